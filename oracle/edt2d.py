"""The decoupled 2D extended-diffraction-tomography method, written out plainly in FP64.

Discrete reading of the paper's continuous derivation (Section "Two dimensions"):

* Lateral grid x_i = i dx, i < N, periodic with L = N dx.  Sources and receivers sit on
  every grid point at z = 0.  Wavenumbers k_n = 2 pi n'/L with n' = n (n <= N/2) or n - N.
  Periodicity is the discrete form of "treat the survey as infinite" after the complex
  frequency omega -> omega + i eps (the a sinc -> pi delta step); it also records every
  offset, so the aperture sinc of eq. M reduces to a delta.
* Depths z_j = z0 + (j + 1/2) dz (midpoint rule for the depth integral of eq. Born).
* Born data (eq. Born, omega^2 -> omega~^2):
      D(is, ir) = omega~^2 dx dz sum_x sum_j G(x_ir - x, z_j) V(x, z_j) G(x - x_is, z_j).
* Data transform (the Fourier transform over m and h, on the shot/receiver grid):
      D2(p, q) = sum_is sum_ir D(is, ir) exp(-i k_p x_ir) exp(+i k_q x_is).
  For midpoint wavenumber index m (k_m = k_p - k_q) this gives the decoupled system of
  eqs. DMV and M,
      D2(p, p - m) = sum_j M[(omega, p), j] Vhat(k_m, z_j),
      M[(omega, p), j] = (omega~^2 dz / dx) g(k_p, z_j) g(k_{p-m}, z_j),
  with Vhat(k, z) = sum_x V(x, z) exp(-i k x).
* Hermitian split (eq. Split): the row (p, q) of k_m and the row (q, p) of -k_m carry the
  same M, so with d_+ = (D2(p,q) + D2(q,p))/2 and d_- = (D2(p,q) - D2(q,p))/(2i),
      M Re Vhat = d_+,   M Im Vhat = d_-,
  solved for real unknowns for 0 <= m <= N/2; Vhat(-k_m) = conj Vhat(k_m) (eq. VSym).  At
  the self-paired m = 0 and m = N/2 only the real part is solved (Im Vhat = 0 there).
* Solve: the paper uses a truncated SVD; this project uses damped least squares
  (zeroth-order Tikhonov, which the paper's Discussion names as the next step):
      min ||Ahat x - dhat||^2 + lam ||x||^2,  Ahat = [Re M; Im M],  lam = alpha ||Ahat||_F^2,
  by Householder QR of [Ahat; sqrt(lam) I].  No normal matrix is formed.
* Rows whose two legs are evanescent in the slowest layer (|k| c_min >= cutoff * 2 pi f)
  are dropped (integer test |n'| c_min < (cutoff f) L; cutoff <= 0 keeps every row).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

from .green import green_layered


# ----------------------------------------------------------------------------- geometry
def signed_index(N):
    """n' = n for n <= N/2, n - N otherwise."""
    n = np.arange(N)
    return np.where(n <= N // 2, n, n - N)


def lateral_wavenumbers(N, dx):
    """k_n = 2 pi n' / (N dx)."""
    return 2 * np.pi * signed_index(N) / (N * dx)


def depths(nz, dz, z0):
    """z_j = z0 + (j + 1/2) dz."""
    return z0 + (np.arange(nz) + 0.5) * dz


def complex_omega(freq_hz, eps):
    """omega~ = 2 pi f + i eps (Section "Two dimensions", the complex-frequency step)."""
    return 2 * np.pi * np.asarray(freq_hz, dtype=np.float64) + 1j * eps


def green_table(wl):
    """g(k_n, z_j; omega~_f) for every frequency f, lateral index n and depth j: [f][n][j]."""
    k = lateral_wavenumbers(wl.nx, wl.dx)
    z = depths(wl.nz, wl.dz, wl.z0)
    om = complex_omega(wl.freq_hz, wl.eps)
    return np.stack([green_layered(o, k, z, wl.layer_top, wl.layer_vel) for o in om])


def born_scale(wl):
    """s_f = omega~_f^2 dz / dx, the prefactor of M in the discrete model."""
    return complex_omega(wl.freq_hz, wl.eps) ** 2 * wl.dz / wl.dx


# ----------------------------------------------------------------------------- rows
def kept_rows(wl, m):
    """Rows (f, p) of the k_m system that survive the evanescent cut, in (f, p) order."""
    N = wl.nx
    ns = signed_index(N)
    L = N * wl.dx
    cmin = float(np.min(wl.layer_vel))
    p = np.arange(N)
    q = (p - m) % N
    rows = []
    for f, fr in enumerate(wl.freq_hz):
        if wl.cutoff > 0:
            lim = (wl.cutoff * float(fr)) * L
            keep = (np.abs(ns[p]).astype(np.float64) * cmin < lim) & \
                   (np.abs(ns[q]).astype(np.float64) * cmin < lim)
        else:
            keep = np.ones(N, dtype=bool)
        rows.extend((f, int(pp)) for pp in p[keep])
    return np.array(rows, dtype=np.int64).reshape(-1, 2)


def kernel_rows(wl, m, rows, g=None):
    """M[(f, p), j] = s_f g(k_p, z_j) g(k_{p-m}, z_j) for the given rows (eq. M, delta aperture)."""
    if g is None:
        g = green_table(wl)
    s = born_scale(wl)
    f, p = rows[:, 0], rows[:, 1]
    q = (p - m) % wl.nx
    return s[f, None] * g[f, p, :] * g[f, q, :]


# ----------------------------------------------------------------------------- transforms
def data_transform(D):
    """D2[f](p, q) = sum_is sum_ir D[f](is, ir) exp(-i k_p x_ir) exp(+i k_q x_is)."""
    D = np.asarray(D, dtype=np.complex128)
    N = D.shape[-1]
    X = np.fft.fft(D, axis=2)                 # over ir, sign -:   X[f][is][p]
    Y = np.fft.ifft(X, axis=1) * N            # over is, sign +:   Y[f][q][p]
    return np.transpose(Y, (0, 2, 1))         # [f][p][q]


def split_rhs(D2, m, rows):
    """d_+ and d_- of eq. Split for the rows of k_m (pairing row (p, q) with (q, p) of -k_m)."""
    N = D2.shape[1]
    f, p = rows[:, 0], rows[:, 1]
    q = (p - m) % N
    a = D2[f, p, q]
    b = D2[f, q, p]
    return 0.5 * (a + b), (a - b) / 2j


def lateral_dft(V):
    """Vhat(k_m, z) = sum_x V(x, z) exp(-i k_m x): [m][j]."""
    return np.fft.fft(np.asarray(V, dtype=np.float64), axis=0)


def inverse_lateral_dft(Vhat):
    """V(x, z) = (1/N) sum_m Vhat(k_m, z) exp(+i k_m x) (complex; real for Hermitian Vhat)."""
    return np.fft.ifft(Vhat, axis=0)


# ----------------------------------------------------------------------------- solve
def damped_lstsq(Ahat, dhat, lam):
    """argmin ||Ahat x - dhat||^2 + lam ||x||^2 by Householder QR of [Ahat; sqrt(lam) I].

    ``dhat`` is (rows, nrhs).  numpy's QR (LAPACK Householder) serves as the factorisation.
    """
    n = Ahat.shape[1]
    aug = np.vstack([Ahat, np.sqrt(lam) * np.eye(n)])
    rhs = np.vstack([dhat, np.zeros((n, dhat.shape[1]))])
    Q, R = np.linalg.qr(aug, mode="reduced")
    return solve_triangular(R, Q.T @ rhs, lower=False)


def kz_basis(nz):
    """Orthonormal real basis of depth vectors in order of vertical wavenumber index l:
    the constant, (cos, sin)(2 pi l j / nz) for l = 1 .. ceil(nz/2) - 1, and (-1)^j for even nz.
    Returns (P [nz][nz], l of every column); k_z = 2 pi l / (nz dz)."""
    j = np.arange(nz)
    cols, ls = [np.ones(nz) / np.sqrt(nz)], [0]
    for l in range(1, (nz + 1) // 2):
        cols.append(np.sqrt(2.0 / nz) * np.cos(2 * np.pi * l * j / nz))
        ls.append(l)
        cols.append(np.sqrt(2.0 / nz) * np.sin(2 * np.pi * l * j / nz))
        ls.append(l)
    if nz % 2 == 0:
        cols.append(np.where(j % 2 == 0, 1.0, -1.0) / np.sqrt(nz))
        ls.append(nz // 2)
    return np.stack(cols, axis=1), np.array(ls)


def kz_disk_keep(wl, m, factor):
    """Columns of :func:`kz_basis` inside the disk |(k_m, k_z)| <= factor omega_max / c0 of
    Section "Numerical Examples" (c0 = the slowest reference velocity, omega_max = 2 pi f_max)."""
    K = factor * 2 * np.pi * float(np.max(wl.freq_hz)) / float(np.min(wl.layer_vel))
    km = abs(lateral_wavenumbers(wl.nx, wl.dx)[m])
    _, ls = kz_basis(wl.nz)
    kz = 2 * np.pi * ls / (wl.nz * wl.dz)
    return km ** 2 + kz ** 2 <= K ** 2


def tsvd_lstsq(A, d, tol):
    """Truncated-SVD solution of A x = d (Section "Numerical Examples"): x = V S~^-1 U^T d with
    1/s_j kept for s_j >= sigma; sigma = tol if tol > 0, else |tol| times the largest s_j."""
    U, sv, Vt = np.linalg.svd(A, full_matrices=False)
    if sv.size == 0:
        return np.zeros((A.shape[1], d.shape[1]))
    sigma = tol if tol > 0 else abs(tol) * sv[0]
    inv = np.where((sv >= sigma) & (sv > 0), 1.0 / np.where(sv > 0, sv, 1.0), 0.0)
    return Vt.T @ (inv[:, None] * (U.T @ d))


def solve_wavenumber(wl, D2, m, g=None, return_system=False, solver="damped", tsvd_tol=-1e-3,
                     kz_disk=0.0):
    """Vhat(k_m, z) for one midpoint wavenumber index 0 <= m <= N/2 (eqs. DMV, M, Split).

    ``solver``: "damped" (zeroth-order Tikhonov, lam = alpha ||Ahat||_F^2) or "tsvd" (the
    paper's truncated SVD with tolerance ``tsvd_tol``, see :func:`tsvd_lstsq`).  ``kz_disk`` > 0
    restricts the unknowns to the vertical wavenumbers inside the disk of
    :func:`kz_disk_keep` (x = P c over the kept columns P of :func:`kz_basis`; the damping
    keeps lam of the unrestricted system)."""
    N = wl.nx
    if not 0 <= m <= N // 2:
        raise ValueError("m must lie in [0, N/2]")
    rows = kept_rows(wl, m)
    nz = wl.nz
    if len(rows) == 0:
        empty = np.zeros(nz, dtype=np.complex128)
        return (empty, dict(rows=rows)) if return_system else empty
    A = kernel_rows(wl, m, rows, g)
    dp, dm = split_rhs(D2, m, rows)
    Ahat = np.vstack([A.real, A.imag])
    self_paired = (m == 0) or (2 * m == N)
    cols = [np.concatenate([dp.real, dp.imag])]
    if not self_paired:
        cols.append(np.concatenate([dm.real, dm.imag]))
    dhat = np.stack(cols, axis=1)
    lam = wl.alpha * np.sum(Ahat ** 2)
    if kz_disk > 0:
        P = kz_basis(nz)[0][:, kz_disk_keep(wl, m, kz_disk)]
    else:
        P = np.eye(nz)
    if P.shape[1] == 0:
        x = np.zeros((nz, dhat.shape[1]))
    elif solver == "tsvd":
        x = P @ tsvd_lstsq(Ahat @ P, dhat, tsvd_tol)
    elif solver == "damped":
        x = P @ damped_lstsq(Ahat @ P, dhat, lam)
    else:
        raise ValueError("solver must be 'damped' or 'tsvd'")
    vhat = x[:, 0] + (1j * x[:, 1] if not self_paired else 0.0)
    if return_system:
        return vhat, dict(Ahat=Ahat, dhat=dhat, lam=lam, x=x, rows=rows)
    return vhat


def hermitian_complete(vhat_half, N):
    """Vhat for all m from m = 0..N/2 via Vhat(-k_m) = conj Vhat(k_m) (eq. VSym)."""
    out = np.zeros((N,) + vhat_half.shape[1:], dtype=np.complex128)
    out[: N // 2 + 1] = vhat_half
    for m in range(1, (N + 1) // 2):
        out[N - m] = np.conj(vhat_half[m])
    return out


def invert(wl, D, ms=None, **solve_kw):
    """The whole inversion: data D[f][is][ir] -> (V[x][z] real, Vhat[m][z] for 0 <= m <= N/2).

    With ``ms`` given, only those wavenumbers are solved (the others stay zero) and V is
    not meaningful; used to time or check a subset.  ``solve_kw`` selects the solver variant
    of :func:`solve_wavenumber` (truncated SVD, vertical-wavenumber disk).
    """
    N = wl.nx
    D2 = data_transform(D)
    g = green_table(wl)
    vh = np.zeros((N // 2 + 1, wl.nz), dtype=np.complex128)
    for m in (range(N // 2 + 1) if ms is None else ms):
        vh[m] = solve_wavenumber(wl, D2, m, g, **solve_kw)
    V = inverse_lateral_dft(hermitian_complete(vh, N))
    return V.real, vh


# ----------------------------------------------------------------------------- forward
def forward(wl, V, g=None):
    """Spectral Born data D[f][is][ir] for a real potential V[x][z] (decoupled eq. DMV form).

    D2(p, q) = s_f sum_j g(k_p, z_j) g(k_q, z_j) Vhat(k_p - k_q, z_j), then the inverse of
    :func:`data_transform`.
    """
    N = wl.nx
    if g is None:
        g = green_table(wl)
    s = born_scale(wl)
    vh = lateral_dft(V)                               # [m][j]
    p = np.arange(N)
    D2 = np.zeros((len(wl.freq_hz), N, N), dtype=np.complex128)
    for f in range(len(wl.freq_hz)):
        for m in range(N):
            q = (p - m) % N
            D2[f, p, q] = s[f] * np.sum(g[f, p, :] * g[f, q, :] * vh[m][None, :], axis=1)
    return inverse_data_transform(D2)


def inverse_data_transform(D2):
    """Inverse of :func:`data_transform`: D2[f][p][q] -> D[f][is][ir]."""
    D2 = np.asarray(D2, dtype=np.complex128)
    N = D2.shape[-1]
    Y = np.transpose(D2, (0, 2, 1))                   # [f][q][p]
    X = np.fft.fft(Y, axis=1) / N                     # undo the '+' transform over is
    return np.fft.ifft(X, axis=2)                     # undo the '-' transform over ir


def adjoint(wl, D, g=None):
    """Adjoint of :func:`forward` for <D1, D2> = Re sum conj(D1) D2 and <V1, V2> = sum V1 V2."""
    N = wl.nx
    if g is None:
        g = green_table(wl)
    s = born_scale(wl)
    D = np.asarray(D, dtype=np.complex128)
    E = data_transform(D) / N ** 2                    # adjoint of the inverse transform
    p = np.arange(N)
    vh_adj = np.zeros((N, wl.nz), dtype=np.complex128)
    for f in range(len(wl.freq_hz)):
        for m in range(N):
            q = (p - m) % N
            vh_adj[m] += np.sum(np.conj(s[f] * g[f, p, :] * g[f, q, :]) * E[f, p, q][:, None],
                                axis=0)
    # adjoint of V -> sum_x V exp(-i k_m x), restricted to real V
    return np.real(np.fft.ifft(vh_adj, axis=0) * N)


# ----------------------------------------------------------------------------- adjoint
def invert_adjoint(wl, Vbar, g=None):
    """Dbar = S^T Vbar for the linear map S: D -> V of :func:`invert` (the damped solves'
    matrices depend on the reference only), for <V1, V2> = sum V1 V2 and
    <D1, D2> = Re sum conj(D1) D2.  Every step of :func:`invert` reversed:

    * V = Re (1/N) sum_m Vhat(m) e^{i k_m x} with Vhat(m) = x_+ + i x_- (m = 0..N/2) and its
      conjugate at -m gives xbar(m) = (c_m/N) (Re, Im) sum_x Vbar e^{-i k_m x}, c_m = 1 at the
      self-paired m and 2 otherwise;
    * x = argmin ||Ahat x - dhat||^2 + lam ||x||^2 = (Ahat^T Ahat + lam I)^-1 Ahat^T dhat gives
      dhat_bar = Ahat (Ahat^T Ahat + lam I)^-1 xbar;
    * d_+ = (a + b)/2, d_- = (a - b)/(2i) with a = D2(p, q), b = D2(q, p) give
      abar = dbar_+/2 + (i/2) dbar_-, bbar = dbar_+/2 - (i/2) dbar_-;
    * D2 = T D with T/N unitary per axis gives Dbar = T^H D2bar = N^2 T^-1 D2bar.
    """
    N = wl.nx
    nz = wl.nz
    if g is None:
        g = green_table(wl)
    vb = np.fft.fft(np.asarray(Vbar, dtype=np.float64), axis=0)       # sum_x Vbar e^{-i k_m x}
    D2bar = np.zeros((len(wl.freq_hz), N, N), dtype=np.complex128)
    for m in range(N // 2 + 1):
        rows = kept_rows(wl, m)
        if len(rows) == 0:
            continue
        self_paired = (m == 0) or (2 * m == N)
        c = (1.0 if self_paired else 2.0) / N
        A = kernel_rows(wl, m, rows, g)
        Ahat = np.vstack([A.real, A.imag])
        lam = wl.alpha * np.sum(Ahat ** 2)
        H = Ahat.T @ Ahat + lam * np.eye(nz)
        cols = [c * vb[m].real] + ([] if self_paired else [c * vb[m].imag])
        y = np.linalg.solve(H, np.stack(cols, axis=1))
        db = Ahat @ y                                                 # (2R, ncol)
        R = len(rows)
        dp = db[:R, 0] + 1j * db[R:, 0]
        dm = (db[:R, 1] + 1j * db[R:, 1]) if not self_paired else np.zeros(R, complex)
        abar = 0.5 * dp + 0.5j * dm
        bbar = 0.5 * dp - 0.5j * dm
        f, p = rows[:, 0], rows[:, 1]
        q = (p - m) % N
        np.add.at(D2bar, (f, p, q), abar)
        np.add.at(D2bar, (f, q, p), bbar)
    return N ** 2 * inverse_data_transform(D2bar)
