"""Pins of the finite-aperture / 3D oracle (oracle/edt3d.py) against independent references.

* G(y, z) by FFT against the explicit wavenumber sum;
* the spectral Born forward model against a brute-force space-domain Born sum (eq. Born3D);
* the kernel K(k_m, w, z) by the y-space route against the wavenumber-sum route;
* M(-k_m) = M(k_m) row by row (the symmetry eq. Split needs), the cut's symmetry;
* source/receiver reciprocity of the data (half-offset w -> -w);
* the forward/adjoint dot product;
* with the cut off, the (f, j) system and the (f, w) system have the same solution (the
  window transform is unitary up to a scale, which the damping tracks);
* noise-free recovery, the line-survey special case, and planted mistakes.
"""
import numpy as np
import pytest

import synth
from oracle import edt3d, brute
from oracle.edt2d import complex_omega, depths, damped_lstsq


def tiny(nx=8, ny=6, wx=4, wy=2, nz=3, nf=2, alpha=1e-6, cutoff=1.0):
    tops, vel = synth.layers_gradient_staircase(1500.0, 2500.0, nz * 10.0, 10.0, sub=2)
    return synth.Workload3D("tiny", nx=nx, ny=ny, dx=10.0, dy=12.0, wx=wx, wy=wy,
                            freq_hz=synth.freqs_uniform(nf, 15.0, 40.0), eps=0.15, nz=nz,
                            dz=10.0, z0=0.0, layer_top=tops, layer_vel=vel, alpha=alpha,
                            cutoff=cutoff)


def blobs3(wl, salt=0):
    return synth.perturbation_blobs_3d(synth.rng_for(0, salt), wl.nx, wl.ny, wl.dx, wl.dy,
                                       wl.nz, wl.dz, wl.z0, wl.layer_top, wl.layer_vel,
                                       nblob=3, sigma=25.0, amp=0.05)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def test_green_space_matches_direct_sum():
    wl = tiny()
    g = edt3d.green_grid(wl, 1)
    G = edt3d.green_space(wl, 1, g)
    Gd = brute.green_periodic_2d(g, wl.nx, wl.ny, wl.dx, wl.dy)
    assert rel(G, Gd) < 1e-13


def test_forward_matches_space_domain_born():
    wl = tiny()
    V = blobs3(wl)
    D = edt3d.forward(wl, V)
    for f in range(len(wl.freq_hz)):
        g = edt3d.green_grid(wl, f)
        om = complex_omega(wl.freq_hz[f], wl.eps)
        Db = brute.born_space_domain_3d(om, g, V, wl.nx, wl.ny, wl.dx, wl.dy, wl.dz, wl.wx, wl.wy)
        assert rel(D[f], Db) < 1e-11


@pytest.mark.parametrize("m", [(0, 0), (1, 0), (3, 2), (7, 5), (4, 3)])
def test_kernel_two_routes_agree(m):
    wl = tiny()
    K = edt3d.kernel_offsets(wl, 0)
    Ks = edt3d.kernel_offsets_spectral(wl, 0, m)
    assert rel(K[m[1], m[0]], Ks) < 1e-12


def test_rows_symmetric_in_km_and_cut_symmetric():
    wl = tiny(nx=8, ny=8, wx=4, wy=4)
    M = edt3d.kernel_rows_all(wl, 1)
    for my in range(wl.ny):
        for mx in range(wl.nx):
            nmx, nmy = edt3d.neg(wl, (mx, my))
            a, b = M[my, mx], M[nmy, nmx]
            assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(a))
            assert np.array_equal(edt3d.kept_mask(wl, (mx, my)), edt3d.kept_mask(wl, (nmx, nmy)))


def test_half_offset_reciprocity():
    """Swapping source and receiver maps half-offset w to -w; Born data are reciprocal."""
    wl = tiny(wx=4, wy=4, ny=8)
    D = edt3d.forward(wl, blobs3(wl, 1))
    W = edt3d.window_index(wl.wx)
    for iy, wy in enumerate(edt3d.window_index(wl.wy)):
        for ix, wx in enumerate(W):
            if wx == -wl.wx // 2 or wy == -wl.wy // 2:
                continue
            jy = list(edt3d.window_index(wl.wy)).index(-wy)
            jx = list(W).index(-wx)
            a, b = D[:, :, :, iy, ix], D[:, :, :, jy, jx]
            assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(a))


def test_adjoint_dot_product():
    wl = tiny()
    rng = np.random.default_rng(3)
    V = rng.standard_normal((wl.ny, wl.nx, wl.nz))
    D2 = rng.standard_normal((2, wl.ny, wl.nx, wl.wy, wl.wx)) + 1j * rng.standard_normal(
        (2, wl.ny, wl.nx, wl.wy, wl.wx))
    lhs = np.real(np.vdot(D2, edt3d.forward(wl, V)))
    rhs = float(np.sum(V * edt3d.adjoint(wl, D2)))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_window_transform_leaves_the_solution_unchanged_without_cut():
    wl = tiny(cutoff=0.0, alpha=1e-3)
    rng = np.random.default_rng(5)
    D = rng.standard_normal((2, wl.ny, wl.nx, wl.wy, wl.wx)) + 1j * rng.standard_normal(
        (2, wl.ny, wl.nx, wl.wy, wl.wx))
    _, vh = edt3d.invert(wl, D)
    Dh = np.fft.fft2(D, axes=(1, 2))
    Ks = [edt3d.kernel_offsets(wl, f) for f in range(2)]
    for m in [(0, 0), (2, 1), (5, 3), (4, 3)]:
        mx, my = m
        nmx, nmy = edt3d.neg(wl, m)
        A = np.concatenate([Ks[f][my, mx].reshape(-1, wl.nz) for f in range(2)])
        dpos = np.concatenate([Dh[f, my, mx].ravel() for f in range(2)])
        dneg = np.concatenate([Dh[f, nmy, nmx].ravel() for f in range(2)])
        dp, dm = 0.5 * (dpos + dneg), (dpos - dneg) / 2j
        Ahat = np.vstack([A.real, A.imag])
        lam = wl.alpha * float(np.sum(Ahat ** 2))
        x = damped_lstsq(Ahat, np.stack([np.concatenate([dp.real, dp.imag]),
                                         np.concatenate([dm.real, dm.imag])], axis=1), lam)
        want = x[:, 0] + (0 if edt3d.is_self_paired(wl, m) else 1j * x[:, 1])
        assert rel(vh[my, mx], want) < 1e-10


@pytest.mark.parametrize("name", ["tiny", "line"])
def test_noise_free_recovery(name):
    if name == "tiny":
        wl = tiny(nx=8, ny=8, wx=4, wy=4, nz=4, nf=4, alpha=1e-20, cutoff=0.0)
    else:
        tops, vel = synth.layers_gradient_staircase(1500.0, 2500.0, 60.0, 10.0, sub=2)
        wl = synth.Workload3D("line", nx=16, ny=1, dx=10.0, dy=10.0, wx=8, wy=1,
                              freq_hz=synth.freqs_uniform(6, 10.0, 40.0), eps=0.15, nz=6,
                              dz=10.0, z0=0.0, layer_top=tops, layer_vel=vel, alpha=1e-20,
                              cutoff=0.0)
    V = blobs3(wl, 2)
    D = edt3d.forward(wl, V)
    Vr, vh = edt3d.invert(wl, D)
    assert rel(Vr, V) < 1e-8
    assert np.max(np.abs(np.fft.ifft2(vh, axes=(0, 1)).imag)) < 1e-12 * np.max(np.abs(V))


def test_pair_representatives_cover_the_grid_once():
    wl = tiny(nx=8, ny=6)
    seen = set()
    for m in edt3d.pair_representatives(wl):
        for q in {m, edt3d.neg(wl, m)}:
            assert q not in seen
            seen.add(q)
    assert len(seen) == wl.nx * wl.ny
    assert sum(edt3d.is_self_paired(wl, m) for m in edt3d.pair_representatives(wl)) == 4


def test_cut_counts_match_a_direct_loop():
    """The vectorised cut against a plain loop over (f, j) with the same inequality."""
    wl = synth.preset3d("small_3d")
    cmin = float(np.min(wl.layer_vel))
    for m in [(0, 0), (3, 1), (8, 8), (15, 4)]:
        keep = edt3d.kept_mask(wl, m)
        mx = edt3d.signed(m[0], wl.nx) / (wl.nx * wl.dx)
        my = edt3d.signed(m[1], wl.ny) / (wl.ny * wl.dy)
        for f, fr in enumerate(wl.freq_hz):
            for iy, jy in enumerate(edt3d.window_index(wl.wy)):
                for ix, jx in enumerate(edt3d.window_index(wl.wx)):
                    ok = True
                    for sg in (1, -1):
                        vx = mx + sg * jx / (wl.wx * wl.dx)
                        vy = my + sg * jy / (wl.wy * wl.dy)
                        ok &= cmin * cmin * (vy * vy + vx * vx) < (2 * wl.cutoff * fr) ** 2
                    assert keep[f, iy, ix] == ok


def test_pins_catch_planted_mistakes():
    """A kernel without the midpoint phase exp(-i k_m.w), or with the window transform's
    sign flipped against the data's, fails the symmetry or the recovery pin."""
    wl = tiny(nx=8, ny=8, wx=4, wy=4, nz=4, nf=4, alpha=1e-20, cutoff=0.0)
    K = edt3d.kernel_offsets(wl, 0)
    # (a) dropping the midpoint phase breaks M(-k_m) = M(k_m)
    W = edt3d.window_index(wl.wx)
    ph = np.exp(-2j * np.pi * (np.arange(wl.ny)[:, None, None, None] * edt3d.window_index(wl.wy)[None, None, :, None] / wl.ny
                               + np.arange(wl.nx)[None, :, None, None] * W[None, None, None, :] / wl.nx))
    Kbad = K / ph[..., None]
    m, nm = (1, 2), edt3d.neg(wl, (1, 2))
    assert not np.allclose(Kbad[m[1], m[0]], Kbad[nm[1], nm[0]], rtol=1e-6)
    # (b) a sign error in the window transform of the rows only: recovery fails
    V = blobs3(wl, 2)
    D = edt3d.forward(wl, V)
    orig = edt3d.window_dft

    def flipped(A, axes=(-3, -2)):
        return np.conj(orig(np.conj(A), axes))

    d = edt3d.data_transform(wl, D)
    Ms = [flipped(edt3d.kernel_offsets(wl, f), axes=(2, 3)) for f in range(4)]
    vh = np.zeros((wl.ny, wl.nx, wl.nz), dtype=np.complex128)
    for mm in edt3d.pair_representatives(wl):
        v = edt3d.solve_pair(wl, d, edt3d.kernel_rows_for(wl, mm, Ms), mm)
        vh[mm[1], mm[0]] = v
        n2 = edt3d.neg(wl, mm)
        vh[n2[1], n2[0]] = np.conj(v)
    assert rel(np.fft.ifft2(vh, axes=(0, 1)).real, V) > 1e-3
