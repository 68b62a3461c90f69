"""Gradients of the Born data misfit (line geometry), written out plainly in FP64.

Test infrastructure only: the oracle the GPU gradients are checked against.

The misfit of a model V[x][z] and a layered reference c0 (velocities c_l of fixed layers)
against data D[f][is][ir] is

    J(V, c) = || F(c) V - D ||^2 = sum_f sum_is sum_ir |R(f, is, ir)|^2,   R = F(c) V - D,

with F the spectral Born operator of :func:`oracle.edt2d.forward` (Section "Two dimensions",
eq. Born after the complex-frequency step, decoupled as eqs. DMV and M; every row kept: the
modelling operator has no evanescent cut).  Its gradients:

* with respect to V: grad_V J = 2 F^T R, F^T the adjoint of F for the real inner products
  <V1, V2> = sum V1 V2 and <D1, D2> = Re sum conj(D1) D2 (:func:`oracle.edt2d.adjoint`);
* with respect to the velocity c_l of layer l: dJ/dc_l = 2 <R, (dF/dc_l) V>, where dF/dc_l V
  is the forward model with g(k_p) g(k_q) replaced by its derivative
  dg_p/dc_l g_q + g_p dg_q/dc_l.  The derivative dg/dc_l of the Green's function is
  propagated through the same stable reflectivity recursion the oracle's g uses
  (forward-mode differentiation, one layer at a time).

Every function follows its definition directly; nothing here is shared with the GPU path.
"""
from __future__ import annotations

import numpy as np

from .edt2d import (adjoint, born_scale, complex_omega, depths, forward, lateral_dft,
                    lateral_wavenumbers, inverse_data_transform)
from .green import green_layered, vertical_wavenumber


def misfit(wl, V, D, g=None):
    """J = ||F V - D||^2 summed over every data sample."""
    R = forward(wl, V, g) - np.asarray(D, dtype=np.complex128)
    return float(np.sum(np.abs(R) ** 2))


def grad_V(wl, V, D, g=None):
    """dJ/dV[x][z] = 2 F^T (F V - D)."""
    R = forward(wl, V, g) - np.asarray(D, dtype=np.complex128)
    return 2.0 * adjoint(wl, R, g)


def green_layered_tangent(omega_t, k, z, layer_top, layer_vel, l):
    """(g, dg/dc_l) for arrays k (any shape) and depths z (1D), by forward-mode
    differentiation of the reflectivity recursion of :func:`oracle.green.green_layered`.

    The only dependence on c_l is through the vertical wavenumber of layer l,
    kappa_l = sqrt(omega~^2/c_l^2 - k^2), with d kappa_l / d c_l = -omega~^2 / (c_l^3 kappa_l).
    Every later quantity carries its derivative by the product and quotient rules.
    """
    tops = np.asarray(layer_top, dtype=np.float64)
    vel = np.asarray(layer_vel, dtype=np.float64)
    J = len(tops)
    k = np.asarray(k, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    kk = k[..., None]
    kap = vertical_wavenumber(omega_t ** 2 / vel ** 2 - kk ** 2)       # (..., J)
    dkap = np.zeros_like(kap)
    dkap[..., l] = -omega_t ** 2 / (vel[l] ** 3 * kap[..., l])
    h = np.diff(tops)

    r = np.zeros(kap.shape, dtype=np.complex128)
    dr = np.zeros_like(r)
    rho = np.zeros_like(r)
    drho = np.zeros_like(r)
    for j in range(J - 2, -1, -1):
        num = 1 - r[..., j + 1]
        den = 1 + r[..., j + 1]
        y = kap[..., j + 1] * num / den
        dy = dkap[..., j + 1] * num / den + kap[..., j + 1] * (-2.0 * dr[..., j + 1]) / den ** 2
        a, b = kap[..., j], y
        rho[..., j] = (a - b) / (a + b)
        drho[..., j] = 2.0 * (b * dkap[..., j] - a * dy) / (a + b) ** 2
        e2 = np.exp(2j * kap[..., j] * h[j])
        r[..., j] = rho[..., j] * e2
        dr[..., j] = drho[..., j] * e2 + rho[..., j] * e2 * 2j * h[j] * dkap[..., j]

    amp = np.zeros_like(kap)
    damp = np.zeros_like(kap)
    amp[..., 0] = 1j / (2 * kap[..., 0])
    damp[..., 0] = -1j * dkap[..., 0] / (2 * kap[..., 0] ** 2)
    for j in range(J - 1):
        e1 = np.exp(1j * kap[..., j] * h[j])
        F = e1 * (1 + rho[..., j]) / (1 + r[..., j + 1])
        dF = (e1 * 1j * h[j] * dkap[..., j] * (1 + rho[..., j]) / (1 + r[..., j + 1])
              + e1 * drho[..., j] / (1 + r[..., j + 1])
              - e1 * (1 + rho[..., j]) * dr[..., j + 1] / (1 + r[..., j + 1]) ** 2)
        amp[..., j + 1] = amp[..., j] * F
        damp[..., j + 1] = damp[..., j] * F + amp[..., j] * dF

    out = np.zeros(k.shape + (len(z),), dtype=np.complex128)
    dout = np.zeros_like(out)
    lay = np.searchsorted(tops, z, side="right") - 1
    for iz, zz in enumerate(z):
        if zz < 0:
            raise ValueError("tangent defined for depths below the source only")
        j = lay[iz]
        d = zz - tops[j]
        P = np.exp(1j * kap[..., j] * d)
        if j == J - 1:
            out[..., iz] = amp[..., j] * P
            dout[..., iz] = damp[..., j] * P + amp[..., j] * 1j * d * dkap[..., j] * P
        else:
            Q = np.exp(1j * kap[..., j] * (2 * h[j] - d))
            out[..., iz] = amp[..., j] * (P + rho[..., j] * Q)
            dout[..., iz] = (damp[..., j] * (P + rho[..., j] * Q)
                             + amp[..., j] * (1j * d * dkap[..., j] * P + drho[..., j] * Q
                                              + rho[..., j] * 1j * (2 * h[j] - d) * dkap[..., j] * Q))
    return out, dout


def green_table_tangent(wl, l):
    """(g, dg/dc_l) tables [f][n][j] over every lateral index n and depth j."""
    k = lateral_wavenumbers(wl.nx, wl.dx)
    z = depths(wl.nz, wl.dz, wl.z0)
    om = complex_omega(wl.freq_hz, wl.eps)
    gs, dgs = [], []
    for o in om:
        g, dg = green_layered_tangent(o, k, z, wl.layer_top, wl.layer_vel, l)
        gs.append(g)
        dgs.append(dg)
    return np.stack(gs), np.stack(dgs)


def forward_tangent(wl, V, g, dg):
    """(dF/dc) V: the forward model of eq. DMV with the row product g_p g_q replaced by
    dg_p g_q + g_p dg_q (data domain [f][is][ir])."""
    N = wl.nx
    s = born_scale(wl)
    vh = lateral_dft(V)
    p = np.arange(N)
    D2 = np.zeros((len(wl.freq_hz), N, N), dtype=np.complex128)
    for f in range(len(wl.freq_hz)):
        for m in range(N):
            q = (p - m) % N
            prod = dg[f, p, :] * g[f, q, :] + g[f, p, :] * dg[f, q, :]
            D2[f, p, q] = s[f] * np.sum(prod * vh[m][None, :], axis=1)
    return inverse_data_transform(D2)


def grad_c(wl, V, D):
    """dJ/dc_l for every layer l: 2 Re sum conj(F V - D) (dF/dc_l) V."""
    out = np.zeros(len(wl.layer_vel))
    R = None
    for l in range(len(wl.layer_vel)):
        g, dg = green_table_tangent(wl, l)
        if R is None:
            R = forward(wl, V, g) - np.asarray(D, dtype=np.complex128)
        out[l] = 2.0 * float(np.real(np.vdot(R, forward_tangent(wl, V, g, dg))))
    return out


def invert_tangent(wl, D, l):
    """(V, dV/dc_l): the damped inversion of :func:`oracle.edt2d.invert` and its derivative with
    respect to the velocity of layer l, by forward-mode differentiation of every step in order.

    The data D do not depend on the reference; the kernel rows do (eq. M, through g), and so
    do the normal matrix and the damping lam = alpha ||Ahat||_F^2.  The set of kept rows is
    held fixed (the evanescent cut is a threshold on the slowest velocity; a derivative sees
    no change of it).  Per midpoint index m, with x the damped least-squares solution of
    Ahat x = dhat:
        (Ahat^T Ahat + lam I) x = Ahat^T dhat,
    differentiated:
        (Ahat^T Ahat + lam I) dx = dAhat^T (dhat - Ahat x) - Ahat^T dAhat x - dlam x,
        dlam = 2 alpha <Ahat, dAhat>_F,
    with dAhat the real and imaginary parts of dA = s_f (dg_p g_q + g_p dg_q).  The system
    for dx is solved with the R factor of the same augmented QR the solution uses
    (R^T R = Ahat^T Ahat + lam I).  Then dV follows from dVhat by the same linear map as V
    from Vhat (eq. VSym and the inverse lateral DFT)."""
    from scipy.linalg import solve_triangular
    from .edt2d import (data_transform, kept_rows, split_rhs, hermitian_complete,
                        inverse_lateral_dft)
    N = wl.nx
    D2 = data_transform(D)
    g, dg = green_table_tangent(wl, l)
    s = born_scale(wl)
    vh = np.zeros((N // 2 + 1, wl.nz), dtype=np.complex128)
    dvh = np.zeros_like(vh)
    for m in range(N // 2 + 1):
        rows = kept_rows(wl, m)
        if len(rows) == 0:
            continue
        f, p = rows[:, 0], rows[:, 1]
        q = (p - m) % N
        A = s[f, None] * g[f, p, :] * g[f, q, :]
        dA = s[f, None] * (dg[f, p, :] * g[f, q, :] + g[f, p, :] * dg[f, q, :])
        Ahat = np.vstack([A.real, A.imag])
        dAhat = np.vstack([dA.real, dA.imag])
        dp, dm = split_rhs(D2, m, rows)
        self_paired = (m == 0) or (2 * m == N)
        cols = [np.concatenate([dp.real, dp.imag])]
        if not self_paired:
            cols.append(np.concatenate([dm.real, dm.imag]))
        dhat = np.stack(cols, axis=1)
        lam = wl.alpha * np.sum(Ahat ** 2)
        dlam = 2.0 * wl.alpha * np.sum(Ahat * dAhat)
        nz = wl.nz
        aug = np.vstack([Ahat, np.sqrt(lam) * np.eye(nz)])
        Q, R = np.linalg.qr(aug, mode="reduced")
        x = solve_triangular(R, Q.T @ np.vstack([dhat, np.zeros((nz, dhat.shape[1]))]), lower=False)
        rhs = dAhat.T @ (dhat - Ahat @ x) - Ahat.T @ (dAhat @ x) - dlam * x
        dx = solve_triangular(R, solve_triangular(R, rhs, trans="T", lower=False), lower=False)
        vh[m] = x[:, 0] + (1j * x[:, 1] if not self_paired else 0.0)
        dvh[m] = dx[:, 0] + (1j * dx[:, 1] if not self_paired else 0.0)
    V = inverse_lateral_dft(hermitian_complete(vh, N)).real
    dV = inverse_lateral_dft(hermitian_complete(dvh, N)).real
    return V, dV


def invert_grad_c(wl, D, Vbar):
    """dL/dc_l = <Vbar, dV/dc_l> for every layer l (L any loss of the inverted model V with
    dL/dV = Vbar), from :func:`invert_tangent`."""
    Vbar = np.asarray(Vbar, dtype=np.float64)
    return np.array([float(np.sum(Vbar * invert_tangent(wl, D, l)[1]))
                     for l in range(len(wl.layer_vel))])


def with_velocities(wl, vel):
    """A copy of the workload with the layer velocities replaced."""
    import copy
    w2 = copy.copy(wl)
    w2.layer_vel = np.asarray(vel, dtype=np.float64).copy()
    return w2
