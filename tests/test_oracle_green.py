"""Pins for the oracle's layered Green's function (CPU only).

Each check compares the reflectivity recursion of :mod:`oracle.green` with something it
does not share code with: textbook closed forms (homogeneous medium: the classical
diffraction-tomography limit; two half-spaces: plane-wave reflection/transmission), the
jump conditions of the defining equation, and an independent finite-volume solve.
"""
import numpy as np
import pytest

from oracle.green import green_layered
from oracle.brute import green_finite_difference

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _kz(w2):
    kz = np.sqrt(complex(w2))
    return -kz if kz.imag < 0 else kz


CASES = [  # (f Hz, eps, k 1/m, c)
    (5.0, 0.15, 0.0, 1500.0),
    (12.0, 0.15, 0.03, 1500.0),
    (40.0, 0.15, 0.16, 1800.0),
    (8.0, 0.15, 0.05, 1500.0),    # evanescent: k > omega / c
    (3.0, 2.0, 0.012, 2500.0),
]


@pytest.mark.parametrize("f,eps,k,c", CASES)
def test_homogeneous_closed_form(f, eps, k, c):
    """One half-space: g = i exp(i kappa |z|) / (2 kappa) (classical DT limit)."""
    om = 2 * np.pi * f + 1j * eps
    z = np.array([-30.0, 0.0, 1.0, 25.0, 333.3, 1500.0])
    kap = _kz(om ** 2 / c ** 2 - k ** 2)
    want = 1j * np.exp(1j * kap * np.abs(z)) / (2 * kap)
    got = green_layered(om, np.array([k]), z, [0.0], [c])[0]
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=0)
    # the same medium cut into several layers of equal velocity
    got3 = green_layered(om, np.array([k]), z, [0.0, 10.0, 300.0, 900.0], [c] * 4)[0]
    np.testing.assert_allclose(got3, want, rtol=1e-12, atol=0)


@pytest.mark.parametrize("f,k", [(5.0, 0.0), (10.0, 0.01), (7.0, 0.02), (3.0, 0.009)])
def test_two_layer_closed_form(f, k):
    """The paper's two-layer reference (1500 over 4000 m/s, interface at 1 km):
    g = (i/2k1)[e^{ik1 z} + R e^{ik1(2zI - z)}] above, (i/2k1) T e^{ik1 zI} e^{ik2(z - zI)} below,
    R = (k1 - k2)/(k1 + k2), T = 1 + R."""
    om = 2 * np.pi * f + 0.15j
    c1, c2, zI = 1500.0, 4000.0, 1000.0
    k1, k2 = _kz(om ** 2 / c1 ** 2 - k ** 2), _kz(om ** 2 / c2 ** 2 - k ** 2)
    R = (k1 - k2) / (k1 + k2)
    T = 1 + R
    z = np.array([5.0, 500.0, 999.0, 1000.0, 1001.0, 2500.0])
    want = np.where(z < zI,
                    1j / (2 * k1) * (np.exp(1j * k1 * z) + R * np.exp(1j * k1 * (2 * zI - z))),
                    1j / (2 * k1) * T * np.exp(1j * k1 * zI) * np.exp(1j * k2 * (z - zI)))
    got = green_layered(om, np.array([k]), z, [0.0, zI], [c1, c2])[0]
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=0)


def test_jump_and_continuity():
    """g is continuous, g' jumps by -1 at the source and is continuous at interfaces."""
    om = 2 * np.pi * 9.0 + 0.15j
    tops, vel = [0.0, 120.0, 260.0, 400.0], [1500.0, 2100.0, 1800.0, 3200.0]
    d = 1e-4
    for k in (0.0, 0.02, 0.05):
        g = lambda z: green_layered(om, np.array([k]), np.atleast_1d(z), tops, vel)[0]
        gp = lambda z: (g(z + d) - g(z - d)) / (2 * d)
        jump = (g(2 * d) - g(d)) / d - (g(-d) - g(-2 * d)) / d
        assert abs(jump[0] + 1.0) < 1e-3
        for t in tops[1:]:
            assert abs(g(t - 1e-9)[0] - g(t)[0]) < 1e-9 * abs(g(t)[0]) + 1e-15
            left = (g(t - d) - g(t - 2 * d)) / d
            right = (g(t + 2 * d) - g(t + d)) / d
            assert abs(left[0] - right[0]) < 1e-3 * abs(gp(t - 10)[0]) + 1e-6


def test_finite_difference_brute_force():
    """Second-order convergence of an independent finite-volume solve to the recursion."""
    tops = [0.0, 100.0, 250.0, 400.0]
    vel = [1500.0, 2200.0, 1900.0, 3500.0]
    zev = np.array([20.0, 100.0, 180.0, 330.0, 480.0])
    for f, k in ((10.0, 0.01), (6.0, 0.0), (15.0, 0.055)):
        om = 2 * np.pi * f + 0.15j
        ref = green_layered(om, np.array([k]), zev, tops, vel)[0]
        errs = []
        sols = []
        for h in (1.0, 0.5, 0.25):
            s = green_finite_difference(om, k, tops, vel, zev, h, -200.0, 600.0)
            sols.append(s)
            errs.append(np.max(np.abs(s - ref)) / np.max(np.abs(ref)))
        order = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
        assert 1.8 < order[0] < 2.2 and 1.8 < order[1] < 2.2, (errs, order)
        rich = (4 * sols[2] - sols[1]) / 3
        assert np.max(np.abs(rich - ref)) / np.max(np.abs(ref)) < 5e-6


def test_even_in_k_and_decay():
    """G~(k) = G~(-k) (Section "Two dimensions") and evanescent decay with depth."""
    om = 2 * np.pi * 20.0 + 0.15j
    tops, vel = [0.0, 300.0], [1500.0, 2500.0]
    z = np.linspace(1, 900, 7)
    k = np.array([0.03, 0.2])
    a = green_layered(om, k, z, tops, vel)
    b = green_layered(om, -k, z, tops, vel)
    np.testing.assert_array_equal(a, b)
    assert np.all(np.diff(np.abs(a[1])) < 0)
