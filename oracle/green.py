"""Reference Green's function g(k, z; omega~) of a laterally invariant layered medium (FP64).

The paper defines the reference Green's function G by the Helmholtz equation of Section
"Two dimensions" (omega^2/c0(z)^2 G + lap G = -delta(x - x0)) and uses its lateral Fourier
transform G~(k, z, omega) (the expansion of G in k).  With the non-symmetric convention
G(x, z) = (1/2 pi) int dk e^{ikx} g(k, z), g solves

    g'' + (omega~^2 / c0(z)^2 - k^2) g = -delta(z),      omega~ = omega + i eps,

with the source at the surface z = 0, outgoing / decaying waves at z -> +-inf, and the top
layer's velocity continued above z = 0 (no free surface, as in the paper's examples).
The paper's G~ equals g / sqrt(2 pi); the global factor cancels between modelling and
inversion.  g depends on k only through k^2, so G~(k) = G~(-k) (Section "Two
dimensions", the evenness used to derive eq. Split).

The paper is silent on how to compute g in layers.  This oracle takes the stable
reflectivity recursion: an upward recursion for the reflection coefficient of the stack
below each interface, then a downward recursion for the downgoing amplitude, in which
every exponential has non-positive growth rate.
"""
from __future__ import annotations

import numpy as np


def vertical_wavenumber(w2_minus_k2):
    """kappa = sqrt(omega~^2/c^2 - k^2) on the branch with Im(kappa) >= 0."""
    kz = np.sqrt(np.asarray(w2_minus_k2, dtype=np.complex128))
    return np.where(kz.imag < 0, -kz, kz)


def green_layered(omega_t, k, z, layer_top, layer_vel):
    """g(k, z; omega~) for arrays k (any shape) and depths z (1D), FP64 complex.

    ``layer_top[0]`` must be 0 (the source depth); layer j spans
    [layer_top[j], layer_top[j+1]) and the last layer is a half-space.  A depth equal to
    an interface belongs to the layer below.  Depths z < 0 lie in the top layer's
    continuation above the source.  Returns an array of shape k.shape + (len(z),).
    """
    tops = np.asarray(layer_top, dtype=np.float64)
    vel = np.asarray(layer_vel, dtype=np.float64)
    J = len(tops)
    if J != len(vel) or tops[0] != 0.0 or np.any(np.diff(tops) <= 0):
        raise ValueError("layer_top must start at 0 and increase; one velocity per layer")
    k = np.asarray(k, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    kk = k[..., None]                                    # (..., 1)
    kap = vertical_wavenumber(omega_t ** 2 / vel ** 2 - kk ** 2)   # (..., J)
    h = np.diff(tops)                                    # (J-1,)

    # upward recursion: r_j = reflection of the stack below, referenced at the top of layer j
    r = np.zeros(kap.shape, dtype=np.complex128)
    rho = np.zeros(kap.shape, dtype=np.complex128)
    for j in range(J - 2, -1, -1):
        y = kap[..., j + 1] * (1 - r[..., j + 1]) / (1 + r[..., j + 1])
        rho[..., j] = (kap[..., j] - y) / (kap[..., j] + y)
        r[..., j] = rho[..., j] * np.exp(2j * kap[..., j] * h[j])

    # downward recursion for the downgoing amplitude; jump condition g'(0+) - g'(0-) = -1
    amp = np.zeros(kap.shape, dtype=np.complex128)
    amp[..., 0] = 1j / (2 * kap[..., 0])
    for j in range(J - 1):
        amp[..., j + 1] = (amp[..., j] * np.exp(1j * kap[..., j] * h[j]) * (1 + rho[..., j])
                           / (1 + r[..., j + 1]))

    out = np.zeros(k.shape + (len(z),), dtype=np.complex128)
    lay = np.searchsorted(tops, z, side="right") - 1
    for iz, zz in enumerate(z):
        if zz < 0:
            # above the source: upgoing wave of amplitude u(0) in the top layer
            out[..., iz] = amp[..., 0] * (1 + r[..., 0]) * np.exp(-1j * kap[..., 0] * zz)
            continue
        j = lay[iz]
        dz = zz - tops[j]
        if j == J - 1:
            out[..., iz] = amp[..., j] * np.exp(1j * kap[..., j] * dz)
        else:
            out[..., iz] = amp[..., j] * (np.exp(1j * kap[..., j] * dz)
                                          + rho[..., j] * np.exp(1j * kap[..., j] * (2 * h[j] - dz)))
    return out
