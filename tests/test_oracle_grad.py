"""Pins of the misfit-gradient oracle (oracle/grad2d.py) against independent references.

* dg/dc_l by forward-mode differentiation against central differences of g itself
  (Richardson-extrapolated, so the difference error is far below the tolerance);
* in a stack of layers of one velocity, sum_l dg/dc_l equals the closed-form derivative of
  the homogeneous Green's function g = i/(2 kappa) exp(i kappa z);
* grad_V J against central differences of J (J is quadratic in V, so the central difference
  is exact up to rounding);
* dJ/dc_l against central differences of J with a step of 1e-3 relative (Richardson);
* planted mistakes (a sign error in d kappa/dc, a derivative kept only inside layer l)
  fail the difference pin.
"""
import numpy as np
import pytest

import synth
from oracle import grad2d
from oracle.edt2d import complex_omega
from oracle.green import green_layered


def tiny(nlayer=3, nx=8, nz=5, nf=2):
    tops = np.arange(nlayer) * 18.0
    vel = np.linspace(1600.0, 2600.0, nlayer)
    return synth.Workload("tiny", nx=nx, dx=10.0, freq_hz=synth.freqs_uniform(nf, 15.0, 35.0),
                          eps=0.15, nz=nz, dz=10.0, z0=0.0, layer_top=tops, layer_vel=vel,
                          alpha=1e-3, cutoff=0.0)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def central(fun, x0, h):
    """Richardson-extrapolated central difference (error O(h^4))."""
    d1 = (fun(x0 + h) - fun(x0 - h)) / (2 * h)
    d2 = (fun(x0 + h / 2) - fun(x0 - h / 2)) / h
    return (4 * d2 - d1) / 3


@pytest.mark.parametrize("l", [0, 1, 3])
def test_green_tangent_matches_differences(l):
    tops = np.array([0.0, 40.0, 95.0, 160.0])
    vel = np.array([1500.0, 2100.0, 1800.0, 3000.0])
    om = complex_omega(22.0, 0.15)
    k = np.array([0.0, 0.01, 0.05, 0.2])
    z = np.array([5.0, 39.0, 41.0, 100.0, 170.0, 400.0])
    _, dg = grad2d.green_layered_tangent(om, k, z, tops, vel, l)

    def g_of(c):
        v = vel.copy()
        v[l] = c
        return green_layered(om, k, z, tops, v)

    want = central(g_of, vel[l], 1e-3 * vel[l])
    assert rel(dg, want) < 1e-7


def test_layer_derivatives_sum_to_homogeneous_closed_form():
    c = 2000.0
    tops = np.array([0.0, 30.0, 70.0, 110.0])
    vel = np.full(4, c)
    om = complex_omega(17.0, 0.15)
    k = np.array([0.0, 0.02, 0.07])
    z = np.array([3.0, 35.0, 90.0, 300.0])
    total = sum(grad2d.green_layered_tangent(om, k, z, tops, vel, l)[1] for l in range(4))
    kap = np.sqrt(om ** 2 / c ** 2 - k[:, None] ** 2 + 0j)
    kap = np.where(kap.imag < 0, -kap, kap)
    dkap = -om ** 2 / (c ** 3 * kap)
    e = np.exp(1j * kap * z[None, :])
    want = (-1j / (2 * kap ** 2) + 1j / (2 * kap) * 1j * z[None, :]) * e * dkap
    assert rel(total, want) < 1e-12


def test_grad_V_matches_differences():
    wl = tiny()
    rng = np.random.default_rng(1)
    V = rng.standard_normal((wl.nx, wl.nz)) * 1e-8
    D = synth.random_data(rng, (2, wl.nx, wl.nx)) * 1e-6
    G = grad2d.grad_V(wl, V, D)
    dV = rng.standard_normal(V.shape) * 1e-8
    fd = (grad2d.misfit(wl, V + dV, D) - grad2d.misfit(wl, V - dV, D)) / 2
    assert abs(fd - np.sum(G * dV)) < 1e-9 * abs(fd)


@pytest.mark.parametrize("l", [0, 2])
def test_grad_c_matches_differences(l):
    wl = tiny()
    rng = np.random.default_rng(2)
    V = synth.perturbation_blobs(rng, wl.nx, wl.dx, wl.nz, wl.dz, wl.z0, wl.layer_top,
                                 wl.layer_vel, nblob=2, sigma=15.0)
    D = synth.random_data(rng, (2, wl.nx, wl.nx)) * 1e-9
    gc = grad2d.grad_c(wl, V, D)

    def J_of(c):
        v = wl.layer_vel.copy()
        v[l] = c
        return grad2d.misfit(grad2d.with_velocities(wl, v), V, D)

    want = central(J_of, wl.layer_vel[l], 1e-3 * wl.layer_vel[l])
    assert abs(gc[l] - want) < 1e-6 * abs(want)


def test_planted_mistakes_fail_the_difference_pin(monkeypatch):
    wl = tiny()
    rng = np.random.default_rng(3)
    V = synth.perturbation_blobs(rng, wl.nx, wl.dx, wl.nz, wl.dz, wl.z0, wl.layer_top,
                                 wl.layer_vel, nblob=2, sigma=15.0)
    D = synth.random_data(rng, (2, wl.nx, wl.nx)) * 1e-9
    l = 1

    def J_of(c):
        v = wl.layer_vel.copy()
        v[l] = c
        return grad2d.misfit(grad2d.with_velocities(wl, v), V, D)

    want = central(J_of, wl.layer_vel[l], 1e-3 * wl.layer_vel[l])
    assert abs(grad2d.grad_c(wl, V, D)[l] - want) < 1e-6 * abs(want)
    orig = grad2d.green_layered_tangent

    def sign_flip(*a):
        g, dg = orig(*a)
        return g, -dg

    monkeypatch.setattr(grad2d, "green_layered_tangent", sign_flip)
    assert abs(grad2d.grad_c(wl, V, D)[l] - want) > 1e-2 * abs(want)

    def inside_only(om, k, z, tops, vel, ll):
        g, dg = orig(om, k, z, tops, vel, ll)
        lay = np.searchsorted(tops, z, side="right") - 1
        return g, np.where((lay == ll)[None, :], dg, 0.0)

    monkeypatch.setattr(grad2d, "green_layered_tangent", inside_only)
    assert abs(grad2d.grad_c(wl, V, D)[l] - want) > 1e-2 * abs(want)


# ---- the inversion's derivative with respect to the reference (dV/dc_l through the damped solve)
def _inv_case(alpha, cutoff, nx=8, nz=5, nf=3, salt=4):
    wl = tiny(nlayer=4, nx=nx, nz=nz, nf=nf)
    wl.alpha = alpha
    wl.cutoff = cutoff
    rng = np.random.default_rng(salt)
    V = synth.perturbation_blobs(rng, wl.nx, wl.dx, wl.nz, wl.dz, wl.z0, wl.layer_top,
                                 wl.layer_vel, nblob=2, sigma=15.0)
    from oracle import edt2d
    D = edt2d.forward(wl, V)
    D = D + 0.1 * np.sqrt(np.mean(np.abs(D) ** 2)) * synth.random_data(rng, D.shape)
    return wl, D


@pytest.mark.parametrize("l,alpha", [(0, 1e-1), (1, 1e-3), (3, 1e-2), (2, 1e-5)])
def test_invert_tangent_matches_differences(l, alpha):
    """dV/dc_l against central differences of the oracle's own inversion (no cut, so the row
    set cannot change with the velocities), at strong and weak damping."""
    from oracle import edt2d
    wl, D = _inv_case(alpha, 0.0)
    V, dV = grad2d.invert_tangent(wl, D, l)
    assert rel(V, edt2d.invert(wl, D)[0]) < 1e-13

    def V_of(c):
        v = wl.layer_vel.copy()
        v[l] = c
        return edt2d.invert(grad2d.with_velocities(wl, v), D)[0]

    want = central(V_of, wl.layer_vel[l], 1e-3 * wl.layer_vel[l])
    assert rel(dV, want) < 1e-6


@pytest.mark.parametrize("l", [1, 3])
def test_invert_grad_c_with_the_cut_matches_differences(l):
    """With the evanescent cut, layers other than the slowest leave the row set unchanged:
    dL/dc_l = <Vbar, dV/dc_l> against central differences of L(c) = <Vbar, V(c)>."""
    from oracle import edt2d
    wl, D = _inv_case(1e-2, 1.0, nx=16, nz=6, nf=4, salt=5)
    assert l != int(np.argmin(wl.layer_vel))
    Vbar = np.random.default_rng(6).standard_normal((wl.nx, wl.nz))
    gc = grad2d.invert_grad_c(wl, D, Vbar)

    def L_of(c):
        v = wl.layer_vel.copy()
        v[l] = c
        return float(np.sum(Vbar * edt2d.invert(grad2d.with_velocities(wl, v), D)[0]))

    want = central(L_of, wl.layer_vel[l], 1e-3 * wl.layer_vel[l])
    assert abs(gc[l] - want) < 1e-6 * abs(want)


def test_invert_tangent_planted_mistake_fails_the_difference_pin(monkeypatch):
    """A derivative of the table with the wrong sign (a plausible slip in the chain rule) is
    caught by the difference pin at the damping where the lam term matters most."""
    from oracle import edt2d
    wl, D = _inv_case(1e-1, 0.0)
    l = 1

    def V_of(c):
        v = wl.layer_vel.copy()
        v[l] = c
        return edt2d.invert(grad2d.with_velocities(wl, v), D)[0]

    want = central(V_of, wl.layer_vel[l], 1e-3 * wl.layer_vel[l])
    orig = grad2d.green_table_tangent

    def half(w, ll):
        g, dg = orig(w, ll)
        return g, 0.5 * dg

    monkeypatch.setattr(grad2d, "green_table_tangent", half)
    assert rel(grad2d.invert_tangent(wl, D, l)[1], want) > 1e-2
