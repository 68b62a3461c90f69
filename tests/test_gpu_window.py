"""GPU parity of the finite-aperture (window) geometry against the FP64 oracle (oracle/edt3d.py).

The mixed path (FP32 kernel-row assembly and data transforms, split BF16x3 tensor-core
Gram, FP64-class Cholesky, one refinement step) is compared with the oracle's QR solution on
the same seeded inputs: V and Vhat to 1e-5 relative L2.  Cases: a 32 x 32 grid with a
4 x 4 window, a 64-point line with a 16-sample aperture, a 64 x 64 grid with an 8 x 8
window and odd depth count, the cut disabled, complex128 data; and the 128 x 128 grid with
the 16 x 16 window of the batched 3D workload (two of its frequencies, 200 depths), checked
on sampled pairs whose oracle rows come from the wavenumber-sum route.
"""
import numpy as np
import pytest

import synth
from oracle import edt3d
from tests.gpu_helpers import rel_l2, dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def workload(nx, ny, wx, wy, nf, nz, alpha=1e-4, cutoff=1.0, fmin=10.0, fmax=40.0, dx=10.0):
    tops, vel = synth.layers_gradient_staircase(1500.0, 3000.0, nz * 10.0, 10.0, sub=2)
    return synth.Workload3D("t", nx=nx, ny=ny, dx=dx, dy=dx, wx=wx, wy=wy,
                            freq_hz=synth.freqs_uniform(nf, fmin, fmax), eps=0.15, nz=nz,
                            dz=10.0, z0=0.0, layer_top=tops, layer_vel=vel, alpha=alpha,
                            cutoff=cutoff)


def born_data(wl, salt):
    V = synth.perturbation_blobs_3d(synth.rng_for(0, salt), wl.nx, wl.ny, wl.dx, wl.dy, wl.nz,
                                    wl.dz, wl.z0, wl.layer_top, wl.layer_vel, nblob=3,
                                    sigma=30.0, amp=0.05)
    D = edt3d.forward(wl, V)
    return D + synth.noise_snr(synth.rng_for(0, salt + 100), D, 20.0)


def solver(wl, **kw):
    from paper_0905_0238_gb300 import Config, Solver
    return Solver(Config.from_workload(wl, **kw))


@pytest.mark.parametrize("case", ["grid32_w4", "line64_w16", "grid64_w8_oddnz", "nocut_c128"])
def test_window_matches_oracle(case):
    if case == "grid32_w4":
        wl = workload(32, 32, 4, 4, nf=4, nz=12)
    elif case == "line64_w16":
        wl = workload(64, 1, 16, 1, nf=8, nz=16, fmin=5.0)
    elif case == "grid64_w8_oddnz":
        wl = workload(64, 64, 8, 8, nf=3, nz=13)
    else:
        wl = workload(32, 32, 2, 2, nf=3, nz=10, cutoff=0.0, alpha=1e-3)
    D = born_data(wl, salt=7)
    V_or, vh_or = edt3d.invert(wl, D)
    s = solver(wl)
    if case == "nocut_c128":
        V = s.invert(dev(D)).cpu().numpy()
    else:
        V = s.invert(dev(D.astype(np.complex64)), out_dtype=torch.float32).cpu().numpy()
    st = s.stats()
    assert st.n_notpd == 0 and st.n_nonfinite == 0
    reps = edt3d.pair_representatives(wl)
    vh = s.vhat().cpu().numpy()
    want = np.stack([vh_or[m[1], m[0]] for m in reps])
    assert V.shape == (wl.ny, wl.nx, wl.nz)
    assert rel_l2(vh, want) < 1e-5, rel_l2(vh, want)
    assert rel_l2(V, V_or) < 1e-5, rel_l2(V, V_or)


def test_row_counts_match_the_oracle_cut():
    wl = workload(32, 32, 4, 4, nf=4, nz=12)
    s = solver(wl)
    want = [int(edt3d.kept_mask(wl, m).sum()) for m in edt3d.pair_representatives(wl)]
    assert list(s.row_counts()) == want


def test_batched_grid_sampled_pairs():
    """128 x 128 midpoints, 16 x 16 half-offsets, 200 depths (two frequencies of the batched
    3D workload), seeded random data; sampled pairs against oracle rows built one by one."""
    wl = synth.preset3d("batched_3d")
    wl.freq_hz = wl.freq_hz[[20, 63]]
    rng = synth.rng_for(2, salt=9)
    D = synth.random_data(rng, (2, wl.ny, wl.nx, wl.wy, wl.wx), np.complex64)
    s = solver(wl)
    s.invert(dev(D), out_dtype=torch.float32)
    st = s.stats()
    assert st.n_notpd == 0 and st.n_nonfinite == 0
    vh = s.vhat().cpu().numpy()
    reps = edt3d.pair_representatives(wl)
    d = edt3d.data_transform(wl, D.astype(np.complex128))
    for idx in (0, 1, 777, 4100, len(reps) - 1):
        m = reps[idx]
        want = edt3d.solve_pair(wl, d, edt3d.kernel_rows_for(wl, m), m)
        assert rel_l2(vh[idx], want) < 1e-5, (m, rel_l2(vh[idx], want))


@pytest.mark.parametrize("alpha,refine", [(1e-3, 1), (1e-4, 2)])
@pytest.mark.parametrize("nx,ny,wx,wy,nf,nz", [
    (64, 64, 8, 4, 3, 12),      # rectangular window: derived rows with WY < WX, two jx per thread
    (32, 32, 4, 2, 4, 10),      # WY = 2: no derived rows
    (64, 64, 16, 8, 2, 9),      # 16 x 8 window, odd depth count
    (128, 1, 8, 1, 4, 16),      # lines of 128 and 512 points
    (512, 1, 4, 1, 3, 12),
])
def test_window_shapes_match_oracle(nx, ny, wx, wy, nf, nz, alpha, refine):
    """More grid and window shapes at alpha = 1e-3 (one refinement step) and 1e-4 (two: the
    window Gram's BF16 hi/lo rows make one step contract by only ~0.2 at that damping; the
    64 x 64 grid with the 8 x 4 window is at 6e-6 after one step, 1.3e-6 after two)."""
    wl = workload(nx, ny, wx, wy, nf=nf, nz=nz, alpha=alpha)
    D = born_data(wl, salt=11)
    V_or, vh_or = edt3d.invert(wl, D)
    s = solver(wl, refine=refine)
    V = s.invert(dev(D.astype(np.complex64)), out_dtype=torch.float32).cpu().numpy()
    st = s.stats()
    assert st.n_notpd == 0 and st.n_nonfinite == 0
    reps = edt3d.pair_representatives(wl)
    want = np.stack([vh_or[m[1], m[0]] for m in reps])
    assert rel_l2(s.vhat().cpu().numpy(), want) < 1e-5
    assert rel_l2(V, V_or) < 1e-5
