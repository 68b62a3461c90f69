"""Pins for the oracle's solver variants of Section "Numerical Examples" (CPU only): the
truncated SVD with tolerance sigma and the restriction of the model to a disk in (k_m, k_z).

The vertical-wavenumber basis is pinned by its orthonormality and by numpy's FFT of its columns;
the disk by the depth spectrum of the solution (no energy outside the kept wavenumbers), by
noise-free recovery of a model inside the disk and by the unrestricted solve when the disk
keeps everything; the truncated SVD by plain least squares (tolerance below every singular
value), by zero (tolerance above all) and by the eigen-decomposition of the normal matrix.
"""
import numpy as np
import pytest

import synth
from oracle import edt2d


def line(nx=16, nz=12, nf=4, alpha=1e-3, dz=15.0, fmax=18.0):
    return synth.Workload("line", nx=nx, dx=20.0, freq_hz=synth.freqs_uniform(nf, 6.0, fmax), eps=0.15,
                          nz=nz, dz=dz, z0=3.0, layer_top=np.array([0.0, 40.0, 95.0]),
                          layer_vel=np.array([1500.0, 1900.0, 2600.0]), alpha=alpha, cutoff=0.0)


@pytest.mark.parametrize("nz", [7, 12])
def test_kz_basis_orthonormal_and_labelled_by_fft(nz):
    P, ls = edt2d.kz_basis(nz)
    np.testing.assert_allclose(P.T @ P, np.eye(nz), atol=1e-13)
    for c in range(nz):
        spec = np.abs(np.fft.fft(P[:, c]))
        lab = np.minimum(np.arange(nz), nz - np.arange(nz))       # |l| of every FFT bin
        assert np.all(spec[lab != ls[c]] < 1e-12)


def data(wl, salt):
    rng = synth.rng_for(0, salt=salt)
    return edt2d.data_transform(synth.random_data(rng, (len(wl.freq_hz), wl.nx, wl.nx)))


def test_disk_keeping_everything_is_the_unrestricted_solve():
    wl = line()
    D2 = data(wl, 31)
    for m in (0, 3, 8):
        a = edt2d.solve_wavenumber(wl, D2, m)
        b = edt2d.solve_wavenumber(wl, D2, m, kz_disk=50.0)
        np.testing.assert_allclose(b, a, rtol=1e-10, atol=1e-12 * np.max(np.abs(a)))


def test_disk_solution_has_no_depth_spectrum_outside_the_disk():
    wl = line(nz=16)
    D2 = data(wl, 32)
    _, ls = edt2d.kz_basis(wl.nz)
    for m in (1, 3, 4):
        keep = edt2d.kz_disk_keep(wl, m, 1.2)
        assert 0 < keep.sum() < wl.nz
        lmax = ls[keep].max()
        v = edt2d.solve_wavenumber(wl, D2, m, kz_disk=1.2)
        for part in (v.real, v.imag):
            spec = np.abs(np.fft.fft(part))
            lab = np.minimum(np.arange(wl.nz), wl.nz - np.arange(wl.nz))
            assert np.all(spec[lab > lmax] <= 1e-12 * max(spec.max(), 1e-300))


def disk_recovery_error(keep_fn):
    """Relative error of the disk-restricted solve recovering, from noise-free data at vanishing
    damping, a model built inside the disk that ``keep_fn`` defines."""
    wl = line(nz=10, nf=6, alpha=1e-16, dz=10.0, fmax=30.0)
    g = edt2d.green_table(wl)
    P, _ = edt2d.kz_basis(wl.nz)
    rng = synth.rng_for(0, salt=33)
    err = 0.0
    for m in (1, 5):
        keep = keep_fn(wl, m, 1.0)
        assert 0 < keep.sum() < wl.nz
        rows = edt2d.kept_rows(wl, m)
        A = edt2d.kernel_rows(wl, m, rows, g)
        x = P[:, keep] @ rng.standard_normal((keep.sum(), 2))   # x_+, x_- inside the disk
        N = wl.nx
        D2 = np.zeros((len(wl.freq_hz), N, N), dtype=np.complex128)
        f, p = rows[:, 0], rows[:, 1]
        q = (p - m) % N
        # d_+ = A x_+ and d_- = A x_- through the pairing (p, q) <-> (q, p) of eq. Split
        D2[f, p, q] = A @ x[:, 0] + 1j * (A @ x[:, 1])
        D2[f, q, p] = A @ x[:, 0] - 1j * (A @ x[:, 1])
        v = edt2d.solve_wavenumber(wl, D2, m, kz_disk=1.0)
        want = x[:, 0] + 1j * x[:, 1]
        err = max(err, np.linalg.norm(v - want) / np.linalg.norm(want))
    return err


def test_disk_recovers_a_model_inside_the_disk():
    assert disk_recovery_error(edt2d.kz_disk_keep) < 1e-7


def test_wavenumber_outside_the_disk_is_zero():
    wl = line(nx=32)
    D2 = data(wl, 34)
    K = 0.3 * 2 * np.pi * wl.freq_hz.max() / wl.layer_vel.min()
    km = np.abs(edt2d.lateral_wavenumbers(wl.nx, wl.dx))
    m = int(np.argmax(km[: wl.nx // 2 + 1] > K))
    assert m > 0 and not edt2d.kz_disk_keep(wl, m, 0.3).any()
    assert np.all(edt2d.solve_wavenumber(wl, D2, m, kz_disk=0.3) == 0)


def test_tsvd_against_least_squares_zero_and_the_normal_matrix():
    wl = line()
    D2 = data(wl, 35)
    for m in (2, 6):
        _, sysd = edt2d.solve_wavenumber(wl, D2, m, return_system=True)
        Ah, dh = sysd["Ahat"], sysd["dhat"]
        sv = np.linalg.svd(Ah, compute_uv=False)
        # tolerance below every singular value: the plain least-squares solution
        x_ls = np.linalg.lstsq(Ah, dh, rcond=None)[0]
        x = edt2d.tsvd_lstsq(Ah, dh, 0.5 * sv[-1])
        np.testing.assert_allclose(x, x_ls, rtol=1e-8, atol=1e-10 * np.abs(x_ls).max())
        # tolerance above all: nothing kept
        assert np.all(edt2d.tsvd_lstsq(Ah, dh, 2 * sv[0]) == 0)
        # a middle tolerance (absolute and relative): eigen-decomposition of Ahat^T Ahat
        sig = np.sqrt(sv[3] * sv[4])
        lam, W = np.linalg.eigh(Ah.T @ Ah)
        keep = lam >= sig ** 2
        x_eig = W[:, keep] @ ((W[:, keep].T @ (Ah.T @ dh)) / lam[keep, None])
        for tol in (sig, -sig / sv[0]):
            x = edt2d.tsvd_lstsq(Ah, dh, tol)
            np.testing.assert_allclose(x, x_eig, rtol=1e-8, atol=1e-9 * np.abs(x_eig).max())
        v = edt2d.solve_wavenumber(wl, D2, m, solver="tsvd", tsvd_tol=sig)
        np.testing.assert_allclose(v, x_eig[:, 0] + 1j * x_eig[:, 1], rtol=1e-8,
                                   atol=1e-9 * np.abs(x_eig).max())


def test_planted_disk_mistake_is_caught(monkeypatch):
    """Dropping the last kept vertical wavenumber breaks recovery of a model inside the disk."""
    good = edt2d.kz_disk_keep

    def one_short(wl, m, factor):
        k = good(wl, m, factor).copy()
        k[np.nonzero(k)[0][-1]] = False
        return k

    monkeypatch.setattr(edt2d, "kz_disk_keep", one_short)
    assert disk_recovery_error(good) > 1e-3
