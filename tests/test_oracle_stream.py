"""Pins for the oracle of the streaming 1D subproblems (CPU only).

A request restating one midpoint wavenumber of a line workload must give the line oracle's
Vhat (itself pinned to brute-force Born, closed forms and dot products); the kernel rows of a
homogeneous reference must equal the closed form -s_f e^{i(kz_p + kz_q) z} / (4 kz_p kz_q);
noise-free data must be recovered at vanishing damping; the result must satisfy the damped
normal equations.  The last test plants mistakes in the oracle and checks that a pin fails.
"""
import numpy as np
import pytest

import synth
from synth import stream
from oracle import edt2d, stream1d


def line(nx=16, nz=6, nf=3, cutoff=0.0, alpha=1e-3):
    return synth.Workload("line", nx=nx, dx=20.0, freq_hz=synth.freqs_uniform(nf, 6.0, 18.0),
                          eps=0.15, nz=nz, dz=15.0, z0=3.0,
                          layer_top=np.array([0.0, 22.0, 47.0]),
                          layer_vel=np.array([1500.0, 1900.0, 2600.0]), alpha=alpha, cutoff=cutoff)


def restated(wl, D2, m):
    rows = edt2d.kept_rows(wl, m)
    dp, dm = edt2d.split_rhs(D2, m, rows)
    return stream.sub_from_line(wl, m, rows, dp, dm)


@pytest.mark.parametrize("cutoff", [0.0, 1.0])
def test_restated_line_wavenumber_matches_line_oracle(cutoff):
    wl = line(cutoff=cutoff)
    rng = synth.rng_for(4, salt=1)
    D2 = edt2d.data_transform(synth.random_data(rng, (len(wl.freq_hz), wl.nx, wl.nx)))
    for m in (1, 3, 7):
        sub = restated(wl, D2, m)
        assert sub.nrow == len(edt2d.kept_rows(wl, m))
        want = edt2d.solve_wavenumber(wl, D2, m)
        got = stream1d.solve(sub)
        np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-12 * np.max(np.abs(want)))


def test_kernel_rows_homogeneous_closed_form():
    c = 1800.0
    rng = synth.rng_for(4, salt=2)
    sub = stream.sub1d_random(rng, nz_range=(7, 7), rows_range=(40, 40), layers_range=(1, 1), N=32)
    sub.layer_top = np.array([0.0])
    sub.layer_vel = np.array([c])
    a = stream1d.kernel_rows(sub)
    om = 2 * np.pi * sub.freq_hz + 1j * sub.eps
    z = sub.z0 + (np.arange(sub.nz) + 0.5) * sub.dz
    f, p, q = sub.rows[:, 0], sub.rows[:, 1], sub.rows[:, 2]
    kz = np.sqrt(om[:, None] ** 2 / c ** 2 - sub.kval[None, :] ** 2 + 0j)
    kz = np.where(kz.imag < 0, -kz, kz)
    kp, kq = kz[f, p], kz[f, q]
    s = om[f] ** 2 * sub.dz / sub.dx
    want = -s[:, None] * np.exp(1j * (kp + kq)[:, None] * z[None, :]) / (4 * kp * kq)[:, None]
    np.testing.assert_allclose(a, want, rtol=1e-12, atol=0)


def test_noise_free_recovery_at_vanishing_damping():
    rng = synth.rng_for(4, salt=3)
    sub = stream.sub1d_random(rng, nz_range=(5, 5), rows_range=(200, 200), layers_range=(4, 4),
                              N=32, dz=20.0, fmin=10.0, fmax=40.0, alpha=1e-16)   # cond(Ahat) ~ 7
    x = rng.standard_normal((sub.nz, 2))
    a = stream1d.kernel_rows(sub)
    sub.data = a @ x                                   # d_+- = a x_+- (complex rows, real x)
    got = stream1d.solve(sub)
    np.testing.assert_allclose(got, x[:, 0] + 1j * x[:, 1], rtol=1e-8, atol=1e-8)


def test_solution_satisfies_damped_normal_equations():
    rng = synth.rng_for(4, salt=4)
    sub = stream.sub1d_random(rng, nz_range=(20, 20), rows_range=(150, 150), layers_range=(7, 7), N=64)
    Ahat, dhat, lam = stream1d.system(sub)
    v = stream1d.solve(sub)
    x = np.stack([v.real, v.imag], axis=1)
    res = Ahat.T @ (dhat - Ahat @ x) - lam * x
    assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(Ahat.T @ dhat)
    assert lam == pytest.approx(sub.alpha * np.sum(np.abs(stream1d.kernel_rows(sub)) ** 2), rel=1e-12)


def test_generator_shapes():
    subs = stream.stream_requests(16, salt=5)
    for s in subs:
        assert 64 <= s.nz <= 512 and 128 <= s.nrow <= 4096 and 5 <= len(s.layer_top) <= 30
        assert s.rows.min() >= 0 and s.rows[:, 0].max() < len(s.freq_hz)
        assert s.rows[:, 1:].max() < len(s.kval) and np.all(s.kval >= 0)
        assert s.data.shape == (s.nrow, 2) and s.data.dtype == np.complex64
    sizes, t = stream.burst_schedule(4096, rate_hz=100.0)
    assert sizes.sum() == 4096 and sizes[:-1].min() >= 32 and sizes.max() <= 512
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)


def test_planted_mistakes_are_caught(monkeypatch):
    """A dropped prefactor or the two legs on the same wavenumber break the line restatement."""
    wl = line()
    rng = synth.rng_for(4, salt=6)
    D2 = edt2d.data_transform(synth.random_data(rng, (len(wl.freq_hz), wl.nx, wl.nx)))
    m = 3
    sub = restated(wl, D2, m)
    want = edt2d.solve_wavenumber(wl, D2, m)
    good = stream1d.kernel_rows

    def no_prefactor(s):
        om = edt2d.complex_omega(s.freq_hz, s.eps)
        return good(s) / (om ** 2 * s.dz / s.dx)[s.rows[:, 0], None]

    def same_leg(s):
        s2 = stream.Sub1D(**{**s.__dict__, "rows": np.stack([s.rows[:, 0], s.rows[:, 1], s.rows[:, 1]], 1)})
        return good(s2)

    for bad in (no_prefactor, same_leg):
        monkeypatch.setattr(stream1d, "kernel_rows", bad)
        got = stream1d.solve(sub)
        assert np.linalg.norm(got - want) > 1e-3 * np.linalg.norm(want)
    monkeypatch.setattr(stream1d, "kernel_rows", good)
    np.testing.assert_allclose(stream1d.solve(sub), want, rtol=1e-10, atol=1e-12 * np.max(np.abs(want)))
