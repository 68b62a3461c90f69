"""Finite-aperture and 3D extended diffraction tomography, written out plainly in FP64.

Test infrastructure only: the tests, the smoke check and the benchmark's CPU baseline may
use this module; the library never does.

Discrete reading of Section "A practical 3D geometry" together with eq. M (whose aperture
sinc this form keeps), on a periodic lateral grid:

* Midpoint grid (mx, my), nx x ny points of spacing dx, dy (L_x = nx dx, L_y = ny dy);
  wavenumbers k_a = 2 pi (a_x'/L_x, a_y'/L_y) with signed indices a'.
* Recorded half-offsets: the window w in [-wx/2, wx/2) x [-wy/2, wy/2) (grid steps), the
  source at m - w and the receiver at m + w.  ny = 1, wy = 1 is a 2D line with a finite
  aperture of wx half-offsets.
* Periodic Green's function: G(y, z) = (1/(L_x L_y)) sum_a exp(i k_a.y) g(|k_a|, z), with g
  the 1D Green's function of the layered reference (oracle.green).
* Born data (eq. Born3D, omega^2 -> omega~^2, midpoint rule in depth):
      D(f, m, w) = omega~^2 dx dy dz sum_j sum_x G(m + w - x, z_j) V(x, z_j) G(x - m + w, z_j).
* Transform over midpoints, then the window transform over half-offsets:
      Dhat(k_m; f, w) = sum_m exp(-i k_m.m) D(f, m, w),
      d(k_m; f, j)   = sum_w exp(-2 pi i j.w / W) Dhat(k_m; f, w)   (j signed, k_h = 2 pi j/(W dx)).
* Decoupled system (eq. DMV): Dhat(k_m; f, w) = sum_j K(k_m, w, z_j) Vhat(k_m, z_j) with
      K(k_m, w, z) = omega~^2 dx dy dz sum_y exp(i k_m.(y - w)) G(2w - y, z) G(y, z),
  and the rows of the (f, j) system are M(k_m; f, j, z) = sum_w exp(-2 pi i j.w/W) K(k_m, w, z):
  the window's Dirichlet kernel is the discrete form of the sinc in eq. M.
* M(-k_m) = M(k_m) row by row, so the split of eq. Split applies per row (f, j):
  d_+ = (d(k_m) + d(-k_m))/2, d_- = (d(k_m) - d(-k_m))/(2i); one real damped least-squares
  problem per pair {k_m, -k_m}; at the four self-paired points only the real part.
* Cut: row (f, j) of k_m is kept iff both nominal legs (k_m +- k_h)/2 propagate in the
  slowest layer: c_min^2 ((m_x'/L_x +- j_x/(wx dx))^2 + (m_y'/L_y +- j_y/(wy dy))^2) < (2 cutoff f)^2
  for both signs (cutoff <= 0 keeps every row).
* Solve: damped least squares by Householder QR, lam = alpha tr(Ahat^T Ahat) (as in 2D).
"""
from __future__ import annotations

import numpy as np

from .green import green_layered
from .edt2d import complex_omega, depths, damped_lstsq


# ----------------------------------------------------------------------------- geometry
def signed(n, N):
    """Signed index of n in Z_N: n for n <= N/2, n - N otherwise."""
    n = np.asarray(n)
    return np.where(n <= N // 2, n, n - N)


def window_index(W):
    """The signed half-offsets (or offset wavenumber indices) of a window of W samples."""
    return np.arange(W) - W // 2


def grid_wavenumbers(wl):
    """kx [nx], ky [ny] (rad/m) of the periodic midpoint grid."""
    kx = 2 * np.pi * signed(np.arange(wl.nx), wl.nx) / (wl.nx * wl.dx)
    ky = 2 * np.pi * signed(np.arange(wl.ny), wl.ny) / (wl.ny * wl.dy)
    return kx, ky


def green_grid(wl, f):
    """g(|k_a|, z_j) on the full grid for frequency index f: [ny][nx][nz]."""
    kx, ky = grid_wavenumbers(wl)
    kabs = np.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)
    om = complex_omega(wl.freq_hz[f], wl.eps)
    return green_layered(om, kabs, depths(wl.nz, wl.dz, wl.z0), wl.layer_top, wl.layer_vel)


def green_space(wl, f, g=None):
    """G(y, z_j) = (1/(L_x L_y)) sum_a exp(i k_a.y) g(|k_a|, z_j): [ny][nx][nz]."""
    if g is None:
        g = green_grid(wl, f)
    # numpy's ifft2 carries 1/(nx ny); (nx ny)/(L_x L_y) = 1/(dx dy)
    return np.fft.ifft2(g, axes=(0, 1)) / (wl.dx * wl.dy)


def born_scale3d(wl, f):
    """omega~^2 dx dy dz."""
    om = complex_omega(wl.freq_hz[f], wl.eps)
    return om ** 2 * wl.dx * wl.dy * wl.dz


# ----------------------------------------------------------------------- kernel rows
def kernel_offsets(wl, f, G=None):
    """K(k_m, w, z) for every midpoint wavenumber and half-offset: [my][mx][wy][wx][nz].

    For each half-offset w the product S_w(y) = G(2w - y) G(y) is summed against
    exp(i k_m.y) for all k_m at once (numpy's inverse FFT), then the factor exp(-i k_m.w).
    """
    if G is None:
        G = green_space(wl, f)
    ny, nx = wl.ny, wl.nx
    wxs, wys = window_index(wl.wx), window_index(wl.wy)
    yy, xx = np.arange(ny), np.arange(nx)
    c = born_scale3d(wl, f)
    K = np.zeros((ny, nx, wl.wy, wl.wx, wl.nz), dtype=np.complex128)
    mphase_y = np.exp(-2j * np.pi * np.outer(np.arange(ny), wys) / ny)   # [my][wy]
    mphase_x = np.exp(-2j * np.pi * np.outer(np.arange(nx), wxs) / nx)   # [mx][wx]
    for iy, wy in enumerate(wys):
        for ix, wx in enumerate(wxs):
            Gr = G[(2 * wy - yy) % ny][:, (2 * wx - xx) % nx]          # G(2w - y)
            S = Gr * G
            T = np.fft.ifft2(S, axes=(0, 1)) * (nx * ny)               # sum_y e^{+i k_m.y} S
            K[:, :, iy, ix, :] = c * T * (mphase_y[:, iy][:, None, None] * mphase_x[:, ix][None, :, None])
    return K


def kernel_offsets_spectral(wl, f, m, g=None):
    """K(k_m, w, z) for one midpoint index m = (mx, my) by the wavenumber sum

        K = omega~^2 dz / (nx ny dx dy) sum_a g(|k_a|) g(|k_a + k_m|) exp(-i (2 k_a + k_m).w),

    an independent route to :func:`kernel_offsets` (it never forms G).  Returns [wy][wx][nz].
    """
    if g is None:
        g = green_grid(wl, f)
    mx, my = m
    ny, nx = wl.ny, wl.nx
    ay, ax = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    g_shift = g[(ay + my) % ny, (ax + mx) % nx]                          # g(|k_a + k_m|)
    P = g * g_shift                                                     # [ny][nx][nz]
    om = complex_omega(wl.freq_hz[f], wl.eps)
    c = om ** 2 * wl.dz / (nx * ny * wl.dx * wl.dy)
    out = np.zeros((wl.wy, wl.wx, wl.nz), dtype=np.complex128)
    for iy, wy in enumerate(window_index(wl.wy)):
        for ix, wx in enumerate(window_index(wl.wx)):
            ph = np.exp(-2j * np.pi * ((2 * ay + my) * wy / ny + (2 * ax + mx) * wx / nx))
            out[iy, ix] = c * np.einsum("yx,yxz->z", ph, P)
    return out


def window_dft(A, axes=(-3, -2)):
    """sum_w exp(-2 pi i j.w / W) A[..., w, ...] over the two half-offset axes (signed j, w).

    The default axes are those of K [..][wy][wx][nz]; the result is indexed by (jy, jx).
    """
    A = np.asarray(A)
    out = A
    for ax in axes:
        W = A.shape[ax]
        idx = window_index(W)
        F = np.exp(-2j * np.pi * np.outer(idx, idx) / W)                 # [j][w]
        out = np.moveaxis(np.tensordot(F, np.moveaxis(out, ax, 0), axes=(1, 0)), 0, ax)
    return out


def kernel_rows_all(wl, f, G=None):
    """M(k_m; f, j, z) for every k_m: [my][mx][jy][jx][nz]."""
    return window_dft(kernel_offsets(wl, f, G), axes=(2, 3))


# ------------------------------------------------------------------------------ data
def data_transform(wl, D):
    """D[f][my][mx][wy][wx] -> d[f][my][mx][jy][jx] (midpoint DFT, then window DFT)."""
    Dh = np.fft.fft2(np.asarray(D, dtype=np.complex128), axes=(1, 2))   # sum_m e^{-i k_m.m}
    return window_dft(Dh, axes=(3, 4))


def kept_mask(wl, m):
    """Boolean [nf][jy][jx]: rows (f, j) of midpoint index m = (mx, my) kept by the cut."""
    nf = len(wl.freq_hz)
    if wl.cutoff <= 0:
        return np.ones((nf, wl.wy, wl.wx), dtype=bool)
    cmin = float(np.min(wl.layer_vel))
    mx, my = m
    mxs = float(signed(mx, wl.nx)) / (wl.nx * wl.dx)
    mys = float(signed(my, wl.ny)) / (wl.ny * wl.dy)
    jx = window_index(wl.wx).astype(np.float64) / (wl.wx * wl.dx)
    jy = window_index(wl.wy).astype(np.float64) / (wl.wy * wl.dy)
    lim = (2.0 * wl.cutoff * np.asarray(wl.freq_hz, dtype=np.float64)) ** 2      # [nf]
    keep = np.ones((nf, wl.wy, wl.wx), dtype=bool)
    for sg in (1.0, -1.0):
        vx = mxs + sg * jx                                               # [jx]
        vy = mys + sg * jy                                               # [jy]
        q = (cmin * cmin) * (vy[:, None] ** 2 + vx[None, :] ** 2)
        keep &= q[None, :, :] < lim[:, None, None]
    return keep


def pair_representatives(wl):
    """One midpoint index of every pair {m, -m}: (mx, my) with my in [0, ny/2] and, on the
    rows my = 0 and my = ny/2, mx in [0, nx/2].  Self-paired points come first in each row."""
    reps = []
    for my in range(wl.ny // 2 + 1):
        if my == 0 or 2 * my == wl.ny:
            reps += [(mx, my) for mx in range(wl.nx // 2 + 1)]
        else:
            reps += [(mx, my) for mx in range(wl.nx)]
    return reps


def is_self_paired(wl, m):
    mx, my = m
    return (-mx) % wl.nx == mx and (-my) % wl.ny == my


def neg(wl, m):
    return ((-m[0]) % wl.nx, (-m[1]) % wl.ny)


def solve_pair(wl, d, Mrows, m, return_system=False):
    """Vhat(k_m, z) for one pair representative m from d [nf][my][mx][jy][jx] and the kernel
    rows Mrows[f] = M(k_m; f, j, z) [nf][jy][jx][nz]."""
    keep = kept_mask(wl, m)
    nz = wl.nz
    if not keep.any():
        empty = np.zeros(nz, dtype=np.complex128)
        return (empty, dict(rows=0)) if return_system else empty
    A = Mrows[keep]                                                      # [R][nz]
    mx, my = m
    nmx, nmy = neg(wl, m)
    dpos = d[:, my, mx][keep]
    dneg = d[:, nmy, nmx][keep]
    dp = 0.5 * (dpos + dneg)
    dm = (dpos - dneg) / 2j
    Ahat = np.vstack([A.real, A.imag])
    lam = wl.alpha * float(np.sum(Ahat ** 2))
    if is_self_paired(wl, m):
        x = damped_lstsq(Ahat, np.concatenate([dp.real, dp.imag])[:, None], lam)
        vh = x[:, 0].astype(np.complex128)
    else:
        rhs = np.stack([np.concatenate([dp.real, dp.imag]), np.concatenate([dm.real, dm.imag])], axis=1)
        x = damped_lstsq(Ahat, rhs, lam)
        vh = x[:, 0] + 1j * x[:, 1]
    if return_system:
        return vh, dict(rows=int(keep.sum()), Ahat=Ahat, lam=lam, dp=dp, dm=dm)
    return vh


def kernel_rows_for(wl, m, Ms=None):
    """M(k_m; f, j, z) [nf][jy][jx][nz] for one midpoint index (spectral route per f)."""
    nf = len(wl.freq_hz)
    out = np.zeros((nf, wl.wy, wl.wx, wl.nz), dtype=np.complex128)
    for f in range(nf):
        if Ms is not None:
            out[f] = Ms[f][m[1], m[0]]
        else:
            out[f] = window_dft(kernel_offsets_spectral(wl, f, m), axes=(0, 1))
    return out


def invert(wl, D, ms=None):
    """V [ny][nx][nz] (real) and Vhat [ny][nx][nz] from data D[f][my][mx][wy][wx].

    ``ms``: optional subset of pair representatives to solve (others left zero)."""
    d = data_transform(wl, D)
    nf = len(wl.freq_hz)
    Ms = [kernel_rows_all(wl, f) for f in range(nf)]
    vhat = np.zeros((wl.ny, wl.nx, wl.nz), dtype=np.complex128)
    for m in (pair_representatives(wl) if ms is None else ms):
        v = solve_pair(wl, d, kernel_rows_for(wl, m, Ms), m)
        mx, my = m
        nmx, nmy = neg(wl, m)
        vhat[my, mx] = v
        vhat[nmy, nmx] = np.conj(v)
    V = np.fft.ifft2(vhat, axes=(0, 1))                                  # (1/N) sum e^{+i k.x}
    return V.real, vhat


def forward(wl, V):
    """Born data D[f][my][mx][wy][wx] for a real V [ny][nx][nz] (decoupled spectral form)."""
    vh = np.fft.fft2(np.asarray(V, dtype=np.float64), axes=(0, 1))       # sum_x e^{-i k.x}
    nf = len(wl.freq_hz)
    D = np.zeros((nf, wl.ny, wl.nx, wl.wy, wl.wx), dtype=np.complex128)
    for f in range(nf):
        K = kernel_offsets(wl, f)                                        # [my][mx][wy][wx][nz]
        Dh = np.einsum("yxabz,yxz->yxab", K, vh)
        D[f] = np.fft.ifft2(Dh, axes=(0, 1))
    return D


def adjoint(wl, D):
    """Adjoint of :func:`forward` for <D1, D2> = Re sum conj(D1) D2, <V1, V2> = sum V1 V2."""
    nf = len(wl.freq_hz)
    N = wl.nx * wl.ny
    acc = np.zeros((wl.ny, wl.nx, wl.nz), dtype=np.complex128)
    for f in range(nf):
        K = kernel_offsets(wl, f)
        Dh = np.fft.fft2(np.asarray(D[f], dtype=np.complex128), axes=(0, 1)) / N   # adjoint of ifft2
        acc += np.einsum("yxabz,yxab->yxz", np.conj(K), Dh)
    # adjoint of fft2 (real input) = N ifft2, real part
    return (np.fft.ifft2(acc, axes=(0, 1)) * N).real
