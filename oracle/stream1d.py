"""Independent 1D depth subproblems (the streaming workload), written out plainly in FP64.

Test infrastructure: the oracle is only used by the tests, the smoke check and the benchmark's
CPU baseline; nothing on the product path imports it.

A request is the split system of one midpoint wavenumber (eqs. DMV, M and Split of Section
"Two dimensions") standing on its own, with its own reference and depth grid:

* rows (f, p, q): a_r(z_j) = s_f g(|k_p|, z_j; omega~_f) g(|k_q|, z_j; omega~_f), with
  s_f = omega~_f^2 dz / dx (the discrete Born prefactor), g the layered reference Green's
  function (``oracle.green``), z_j = z0 + (j + 1/2) dz;
* Ahat = [Re a; Im a] (2R x nz), dhat_+- = [Re d_+-; Im d_+-];
* x_+- = argmin ||Ahat x - dhat_+-||^2 + lam ||x||^2 with lam = alpha ||Ahat||_F^2, by
  Householder QR of the augmented matrix (no normal matrix is formed);
* the result is Vhat(k_m, z) = x_+ + i x_-.

Pins (tests/test_oracle_stream.py): a request restating one wavenumber of a line workload
gives the line oracle's Vhat for that wavenumber; the homogeneous-reference rows equal the
closed form; noise-free data are recovered at vanishing damping; the solution satisfies the
damped normal equations.
"""
from __future__ import annotations

import numpy as np

from .edt2d import complex_omega, damped_lstsq, depths
from .green import green_layered


def kernel_rows(sub):
    """a[r][j] = s_f g(|k_p|, z_j) g(|k_q|, z_j) for every row (f, p, q) of the request."""
    om = complex_omega(sub.freq_hz, sub.eps)
    z = depths(sub.nz, sub.dz, sub.z0)
    g = np.stack([green_layered(o, sub.kval, z, sub.layer_top, sub.layer_vel) for o in om])
    s = om ** 2 * sub.dz / sub.dx
    f, p, q = sub.rows[:, 0], sub.rows[:, 1], sub.rows[:, 2]
    return s[f, None] * g[f, p, :] * g[f, q, :]


def system(sub):
    """(Ahat, dhat, lam) of the request: the real-stacked rows, both right-hand sides, damping."""
    a = kernel_rows(sub)
    d = np.asarray(sub.data, dtype=np.complex128)
    Ahat = np.vstack([a.real, a.imag])
    dhat = np.vstack([d.real, d.imag])
    lam = sub.alpha * float(np.sum(Ahat ** 2))
    return Ahat, dhat, lam


def solve(sub):
    """Vhat(z) = x_+ + i x_- of one request (complex128, nz)."""
    if sub.rows.shape[0] == 0:
        return np.zeros(sub.nz, dtype=np.complex128)
    Ahat, dhat, lam = system(sub)
    x = damped_lstsq(Ahat, dhat, lam)
    return x[:, 0] + 1j * x[:, 1]
