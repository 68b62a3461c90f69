"""Brute-force references that pin the oracle (tiny sizes only).

* :func:`green_periodic` and :func:`born_space_domain`: the Born integral of eq. Born
  (Section "Two dimensions") summed directly in the space domain on the periodic grid,
  with the Green's function G(x, z) assembled from g(k, z) by an explicit O(N^2) sum over
  wavenumbers.  It shares only g with :mod:`oracle.edt2d`; it does no Fourier transform of
  the data and never forms the decoupled kernel M.
* :func:`green_periodic_2d` and :func:`born_space_domain_3d`: the same for the finite-
  aperture / 3D geometry (eq. Born3D): G(y, z) by an explicit sum over the 2D wavenumber
  grid and the data D(m, w) of every recorded half-offset summed over the whole grid.
* :func:`green_finite_difference`: the 1D Green's-function equation
  g'' + (omega~^2/c0(z)^2 - k^2) g = -delta(z) solved by second-order finite volumes on a
  fine grid, with exact radiation conditions g' = +- i kappa g at the two ends of the
  domain (exact because the medium is homogeneous beyond them).  It shares nothing with
  :mod:`oracle.green`.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_banded


def green_periodic(g_kn, N, dx):
    """G(x_i, z) = (1/L) sum_n exp(i k_n x_i) g(k_n, z), by direct summation: [i][...]."""
    n = np.arange(N)
    ns = np.where(n <= N // 2, n, n - N)
    L = N * dx
    k = 2 * np.pi * ns / L
    x = n * dx
    ph = np.exp(1j * np.outer(x, k))                 # [i][n]
    return np.tensordot(ph, g_kn, axes=(1, 0)) / L


def born_space_domain(omega_t, g_kn_z, V, dx, dz):
    """D(is, ir) = omega~^2 dx dz sum_x sum_j G(x_ir - x, z_j) V(x, z_j) G(x - x_is, z_j).

    ``g_kn_z`` is g(k_n, z_j) [n][j] for one frequency; V is [x][j].
    """
    N = V.shape[0]
    Gp = green_periodic(g_kn_z, N, dx)               # [i][j], periodic in i
    i = np.arange(N)
    D = np.zeros((N, N), dtype=np.complex128)
    for xs in range(N):
        for xr in range(N):
            Gr = Gp[(xr - i) % N, :]                  # G(x_r - x, z)
            Gs = Gp[(i - xs) % N, :]                  # G(x - x_s, z)
            D[xs, xr] = np.sum(Gr * V * Gs)
    return omega_t ** 2 * dx * dz * D


def green_periodic_2d(g_grid, nx, ny, dx, dy):
    """G(y, z) = (1/(L_x L_y)) sum_a exp(i k_a.y) g(|k_a|, z) by direct summation.

    ``g_grid`` is g on the wavenumber grid [ay][ax][...]; returns [yy][yx][...]."""
    ax = np.arange(nx)
    ay = np.arange(ny)
    kx = 2 * np.pi * np.where(ax <= nx // 2, ax, ax - nx) / (nx * dx)
    ky = 2 * np.pi * np.where(ay <= ny // 2, ay, ay - ny) / (ny * dy)
    phx = np.exp(1j * np.outer(ax * dx, kx))          # [yx][ax]
    phy = np.exp(1j * np.outer(ay * dy, ky))          # [yy][ay]
    G = np.einsum("ya,xb,ab...->yx...", phy, phx, g_grid)
    return G / (nx * dx * ny * dy)


def born_space_domain_3d(omega_t, g_grid, V, nx, ny, dx, dy, dz, wx, wy):
    """D(m, w) = omega~^2 dx dy dz sum_x sum_j G(m + w - x, z_j) V(x, z_j) G(x - m + w, z_j)

    for every midpoint m = (mx, my) and half-offset w of the window [-wx/2, wx/2) x
    [-wy/2, wy/2) (source at m - w, receiver at m + w).  ``g_grid`` [ay][ax][j] for one
    frequency; V [y][x][j].  Returns [my][mx][wy][wx]."""
    G = green_periodic_2d(g_grid, nx, ny, dx, dy)     # [yy][yx][j]
    yy, xx = np.arange(ny), np.arange(nx)
    D = np.zeros((ny, nx, wy, wx), dtype=np.complex128)
    for my in range(ny):
        for mx in range(nx):
            for iy, wyv in enumerate(np.arange(wy) - wy // 2):
                for ix, wxv in enumerate(np.arange(wx) - wx // 2):
                    Gr = G[(my + wyv - yy) % ny][:, (mx + wxv - xx) % nx]      # G(m + w - x)
                    Gs = G[(yy - my + wyv) % ny][:, (xx - mx + wxv) % nx]      # G(x - m + w)
                    D[my, mx, iy, ix] = np.sum(Gr * V * Gs)
    return omega_t ** 2 * dx * dy * dz * D


def green_finite_difference(omega_t, k, layer_top, layer_vel, z_eval, h, z_above, z_below):
    """g(k, z_eval) from a finite-volume solve on the grid z_above + i h (i = 0..).

    ``z_above`` < 0 and ``z_below`` > deepest interface; 0, every interface and every
    z_eval must be grid nodes.  At an interface node the coefficient is the mean of the
    two sides (finite-volume integration of the piecewise-constant coefficient).
    """
    tops = np.asarray(layer_top, dtype=np.float64)
    vel = np.asarray(layer_vel, dtype=np.float64)
    n = int(round((z_below - z_above) / h)) + 1
    z = z_above + h * np.arange(n)

    def q_of(zz):
        j = np.clip(np.searchsorted(tops, zz, side="right") - 1, 0, len(vel) - 1)
        return omega_t ** 2 / vel[j] ** 2 - k ** 2

    q = q_of(z).astype(np.complex128)
    on_iface = np.isin(np.round((z - 0.0) / h).astype(np.int64),
                       np.round(tops[1:] / h).astype(np.int64))
    q[on_iface] = 0.5 * (q_of(z[on_iface] - h / 2) + q_of(z[on_iface] + h / 2))

    def kap(c):
        kz = np.sqrt(omega_t ** 2 / c ** 2 - k ** 2 + 0j)
        return -kz if kz.imag < 0 else kz

    k_top, k_bot = kap(vel[0]), kap(vel[-1])
    main = -2.0 / h ** 2 + q
    upper = np.full(n - 1, 1.0 / h ** 2, dtype=np.complex128)
    lower = np.full(n - 1, 1.0 / h ** 2, dtype=np.complex128)
    # ghost-point radiation conditions: g' = -i k_top g at the top, g' = +i k_bot g at the bottom
    upper[0] = 2.0 / h ** 2
    main[0] += 2j * k_top / h
    lower[-1] = 2.0 / h ** 2
    main[-1] += 2j * k_bot / h
    rhs = np.zeros(n, dtype=np.complex128)
    isrc = int(round(-z_above / h))
    rhs[isrc] = -1.0 / h
    ab = np.zeros((3, n), dtype=np.complex128)
    ab[0, 1:] = upper
    ab[1, :] = main
    ab[2, :-1] = lower
    g = solve_banded((1, 1), ab, rhs)
    idx = np.round((np.asarray(z_eval) - z_above) / h).astype(np.int64)
    return g[idx]
