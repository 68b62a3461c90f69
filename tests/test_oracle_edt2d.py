"""Pins for the oracle's decoupled 2D method (CPU only).

The spectral forward model is pinned to a brute-force space-domain Born sum; the
adjoint by dot-product tests; the kernel rows by the homogeneous closed form and the
M(k_m) = M(-k_m) symmetry; the solve by noise-free recovery, by agreement with two other
least-squares routes and by its optimality condition.  The last test plants plausible
mistakes in the oracle and checks that these pins catch them.
"""
import numpy as np
import pytest

import synth
from oracle import edt2d
from oracle.brute import born_space_domain
from oracle.green import green_layered


def tiny(nx=8, nz=4, nf=3, cutoff=0.0, alpha=1e-3, layers=None, dz=15.0, dx=20.0):
    tops, vel = layers if layers is not None else ([0.0, 22.0, 47.0], [1500.0, 1900.0, 2600.0])
    return synth.Workload("tiny", nx=nx, dx=dx, freq_hz=synth.freqs_uniform(nf, 6.0, 18.0),
                          eps=0.15, nz=nz, dz=dz, z0=3.0, layer_top=np.array(tops),
                          layer_vel=np.array(vel), alpha=alpha, cutoff=cutoff)


def test_forward_matches_space_domain_born():
    wl = tiny()
    rng = synth.rng_for(0, salt=11)
    V = rng.standard_normal((wl.nx, wl.nz)) * 1e-8
    D = edt2d.forward(wl, V)
    g = edt2d.green_table(wl)
    om = edt2d.complex_omega(wl.freq_hz, wl.eps)
    for f in range(len(om)):
        Db = born_space_domain(om[f], g[f], V, wl.dx, wl.dz)
        np.testing.assert_allclose(D[f], Db, rtol=1e-11, atol=1e-12 * np.max(np.abs(Db)))
    # source-receiver reciprocity of Born data: D(is, ir) = D(ir, is)
    np.testing.assert_allclose(D, np.transpose(D, (0, 2, 1)), rtol=1e-11, atol=1e-20)


def test_data_transform_is_the_written_dft():
    rng = synth.rng_for(0, salt=12)
    N = 6
    D = synth.random_data(rng, (2, N, N))
    x = np.arange(N)
    k = 2 * np.pi * np.where(x <= N // 2, x, x - N) / N
    want = np.einsum("fsr,pr,qs->fpq", D, np.exp(-1j * np.outer(k, x)), np.exp(1j * np.outer(k, x)))
    np.testing.assert_allclose(edt2d.data_transform(D), want, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(edt2d.inverse_data_transform(edt2d.data_transform(D)), D, atol=1e-13)


def test_forward_adjoint_dot_product():
    wl = tiny(nx=8, nz=5)
    rng = synth.rng_for(0, salt=13)
    V = rng.standard_normal((wl.nx, wl.nz))
    D = synth.random_data(rng, (len(wl.freq_hz), wl.nx, wl.nx))
    lhs = np.real(np.vdot(edt2d.forward(wl, V), D))
    rhs = np.sum(V * edt2d.adjoint(wl, D))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


def test_kernel_rows_homogeneous_closed_form():
    """Homogeneous reference: M = -omega~^2 dz / (4 dx kz_p kz_q) exp(i (kz_p + kz_q) z)."""
    wl = tiny(nx=16, nz=6, layers=([0.0], [1800.0]))
    m = 3
    rows = edt2d.kept_rows(wl, m)
    A = edt2d.kernel_rows(wl, m, rows)
    om = edt2d.complex_omega(wl.freq_hz, wl.eps)
    k = edt2d.lateral_wavenumbers(wl.nx, wl.dx)
    z = edt2d.depths(wl.nz, wl.dz, wl.z0)
    f, p = rows[:, 0], rows[:, 1]
    q = (p - m) % wl.nx
    kz = lambda kk: np.where(np.sqrt(om[f] ** 2 / 1800.0 ** 2 - kk ** 2 + 0j).imag < 0,
                             -np.sqrt(om[f] ** 2 / 1800.0 ** 2 - kk ** 2 + 0j),
                             np.sqrt(om[f] ** 2 / 1800.0 ** 2 - kk ** 2 + 0j))
    kp, kq = kz(k[p]), kz(k[q])
    want = (-om[f] ** 2 * wl.dz / (4 * wl.dx * kp * kq))[:, None] * np.exp(1j * np.outer(kp + kq, z))
    np.testing.assert_allclose(A, want, rtol=1e-12)


def test_kernel_symmetric_in_midpoint_wavenumber():
    """M(k_h, z; k_m) = M(k_h, z; -k_m): row (p, q) of m equals row (q, p) of N - m."""
    wl = tiny(nx=12, nz=5)
    N = wl.nx
    for m in (1, 4, 5):
        rows = np.array([(f, p) for f in range(len(wl.freq_hz)) for p in range(N)])
        A = edt2d.kernel_rows(wl, m, rows)
        Aneg = edt2d.kernel_rows(wl, N - m, rows)
        f, p = rows[:, 0], rows[:, 1]
        q = (p - m) % N
        # in the -k_m system the row with first index q has second index (q + m) % N = p
        np.testing.assert_allclose(A, Aneg[f * N + q], rtol=1e-15, atol=0)


def test_evanescent_cut_symmetric():
    wl = tiny(nx=32, nz=3, cutoff=1.0, dx=30.0)
    N = wl.nx
    for m in range(N // 2 + 1):
        r1 = {tuple(r) for r in edt2d.kept_rows(wl, m)}
        r2 = {(f, (p + m) % N) for f, p in edt2d.kept_rows(wl, (N - m) % N)}
        assert r1 == r2        # the split partner of every kept row is kept


def _recovery_error(wl, V):
    D = edt2d.forward(wl, V)
    Vrec, _ = edt2d.invert(wl, D)
    return np.linalg.norm(Vrec - V) / np.linalg.norm(V)


def test_noise_free_recovery():
    """Noise-free Born data, many rows per unknown, vanishing damping: V is recovered."""
    wl = tiny(nx=8, nz=4, nf=10, alpha=1e-22, cutoff=0.0, dz=12.0)
    rng = synth.rng_for(0, salt=14)
    V = rng.standard_normal((wl.nx, wl.nz)) * 1e-7
    assert _recovery_error(wl, V) < 1e-11


def test_solve_agrees_with_other_least_squares_routes():
    wl = tiny(nx=16, nz=6, nf=4, alpha=1e-3, cutoff=1.0, dx=40.0)
    rng = synth.rng_for(0, salt=15)
    D = synth.random_data(rng, (len(wl.freq_hz), wl.nx, wl.nx))
    D2 = edt2d.data_transform(D)
    for m in (0, 3, 8):
        assert len(edt2d.kept_rows(wl, m)) > 2 * wl.nz
        _, sysd = edt2d.solve_wavenumber(wl, D2, m, return_system=True)
        Ah, dh, lam, x = sysd["Ahat"], sysd["dhat"], sysd["lam"], sysd["x"]
        n = Ah.shape[1]
        x_ne = np.linalg.solve(Ah.T @ Ah + lam * np.eye(n), Ah.T @ dh)
        x_ls = np.linalg.lstsq(np.vstack([Ah, np.sqrt(lam) * np.eye(n)]),
                               np.vstack([dh, np.zeros((n, dh.shape[1]))]), rcond=None)[0]
        np.testing.assert_allclose(x, x_ne, rtol=1e-9, atol=1e-12 * np.max(np.abs(x)))
        np.testing.assert_allclose(x, x_ls, rtol=1e-9, atol=1e-12 * np.max(np.abs(x)))
        grad = Ah.T @ (dh - Ah @ x) - lam * x
        assert np.linalg.norm(grad) <= 1e-12 * np.linalg.norm(Ah.T @ dh)
        assert np.isclose(lam, wl.alpha * np.trace(Ah.T @ Ah), rtol=1e-12)


def test_output_is_real_and_hermitian():
    wl = tiny(nx=16, nz=5, nf=4, alpha=1e-2, cutoff=1.0)
    rng = synth.rng_for(0, salt=16)
    D = synth.random_data(rng, (len(wl.freq_hz), wl.nx, wl.nx))
    V, vh = edt2d.invert(wl, D)
    full = edt2d.hermitian_complete(vh, wl.nx)
    Vc = edt2d.inverse_lateral_dft(full)
    assert np.max(np.abs(Vc.imag)) <= 1e-14 * np.max(np.abs(Vc.real))
    assert abs(vh[0].imag).max() == 0 and abs(vh[wl.nx // 2].imag).max() == 0


def test_pins_catch_planted_mistakes(monkeypatch):
    """Plausible mistakes planted in the oracle make the recovery or Born pins fail."""
    wl = tiny(nx=8, nz=4, nf=10, alpha=1e-22, cutoff=0.0, dz=12.0)
    rng = synth.rng_for(0, salt=17)
    V = rng.standard_normal((wl.nx, wl.nz)) * 1e-7
    assert _recovery_error(wl, V) < 1e-11

    orig_split, orig_rows, orig_scale = edt2d.split_rhs, edt2d.kernel_rows, edt2d.born_scale

    def split_wrong_sign(D2, m, rows):
        a, b = orig_split(D2, m, rows)
        return a, -b
    mutants = {
        "split sign": ("split_rhs", split_wrong_sign),
        "row index": ("kernel_rows", lambda wl_, m, rows, g=None:
                      orig_rows(wl_, (-m) % wl_.nx if m else 1, rows, g)),
        "conjugated kernel": ("kernel_rows", lambda wl_, m, rows, g=None:
                              np.conj(orig_rows(wl_, m, rows, g))),
    }
    for name, (attr, fn) in mutants.items():
        with monkeypatch.context() as mp:
            mp.setattr(edt2d, attr, fn)
            assert _recovery_error(wl, V) > 1e-3, name
    # a dropped omega~^2 cancels in recovery but not against the space-domain Born sum
    with monkeypatch.context() as mp:
        mp.setattr(edt2d, "born_scale", lambda wl_: orig_scale(wl_) /
                   edt2d.complex_omega(wl_.freq_hz, wl_.eps) ** 2)
        D = edt2d.forward(wl, V)
        g = edt2d.green_table(wl)
        om = edt2d.complex_omega(wl.freq_hz, wl.eps)
        Db = born_space_domain(om[0], g[0], V, wl.dx, wl.dz)
        assert not np.allclose(D[0], Db, rtol=1e-6)


@pytest.mark.parametrize("cutoff", [1.0, 0.0])
def test_invert_adjoint_dot_product(cutoff):
    """<S D, Vbar> = Re <D, S^T Vbar>: the inversion is linear in D, and the adjoint is the
    transpose of that linear map (random D and Vbar)."""
    import synth
    tops, vel = synth.layers_gradient_staircase(1500.0, 2500.0, 60.0, 10.0, sub=2)
    wl = synth.Workload("adj", nx=16, dx=10.0, freq_hz=synth.freqs_uniform(4, 10.0, 40.0),
                        eps=0.15, nz=6, dz=10.0, z0=0.0, layer_top=tops, layer_vel=vel,
                        alpha=1e-3, cutoff=cutoff)
    rng = np.random.default_rng(9)
    D = rng.standard_normal((4, 16, 16)) + 1j * rng.standard_normal((4, 16, 16))
    Vbar = rng.standard_normal((16, 6))
    V, _ = edt2d.invert(wl, D)
    Dbar = edt2d.invert_adjoint(wl, Vbar)
    lhs = float(np.sum(V * Vbar))
    rhs = float(np.real(np.vdot(D, Dbar)))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_invert_adjoint_pin_catches_a_row_mismatch(monkeypatch):
    """A planted mistake -- the adjoint dropping the last kept row of every system, as a
    cut evaluated differently from the forward's would -- breaks the dot-product identity."""
    import synth
    tops, vel = synth.layers_gradient_staircase(1500.0, 2500.0, 60.0, 10.0, sub=2)
    wl = synth.Workload("adj", nx=16, dx=10.0, freq_hz=synth.freqs_uniform(4, 10.0, 40.0),
                        eps=0.15, nz=6, dz=10.0, z0=0.0, layer_top=tops, layer_vel=vel,
                        alpha=1e-3, cutoff=1.0)
    rng = np.random.default_rng(9)
    D = rng.standard_normal((4, 16, 16)) + 1j * rng.standard_normal((4, 16, 16))
    Vbar = rng.standard_normal((16, 6))
    V, _ = edt2d.invert(wl, D)
    lhs = float(np.sum(V * Vbar))
    orig = edt2d.kept_rows
    monkeypatch.setattr(edt2d, "kept_rows", lambda w, m: orig(w, m)[:-1])
    rhs = float(np.real(np.vdot(D, edt2d.invert_adjoint(wl, Vbar))))
    assert abs(lhs - rhs) > 1e-6 * abs(lhs)
