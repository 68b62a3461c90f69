"""Every launch shape the autotuner can pick is a code path: each is checked against the FP64
oracle (1e-5 relative L2 on V), and edt_autotune is checked to keep a valid choice and to
leave the result unchanged (the shapes only regroup the same arithmetic).

Line geometry: a 512-wide workload with 41 frequencies and 12 depths (several transform
chunks for every band budget).  Window geometry: a 32 x 32 grid with a 4 x 4 window.
"""
import numpy as np
import pytest

import synth
from oracle import edt2d, edt3d
from tests.gpu_helpers import rel_l2, small_workload, blobs, dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def line_case():
    wl = small_workload(nx=512, nz=12, nf=41, dx=12.5, dz=8.0, fmin=3.0, fmax=60.0, alpha=1e-3)
    V = blobs(wl, salt=4)
    D = edt2d.forward(wl, V)
    D = D + synth.noise_snr(synth.rng_for(0, salt=78), D, 20.0)
    V_or, _ = edt2d.invert(wl, D)
    return wl, np.ascontiguousarray(D.astype(np.complex64)), V_or


@pytest.mark.parametrize("shape", [dict(band_budget_mb=16, band_cols=4, refine_shape=1, overlap=0),
                                   dict(band_budget_mb=32, band_cols=16, refine_shape=2, overlap=1),
                                   dict(band_budget_mb=96, band_cols=8, refine_shape=3, overlap=0)])
def test_line_launch_shapes_match_oracle(line_case, shape):
    from paper_0905_0238_gb300 import Config, Solver, EDT_MIXED
    wl, D, V_or = line_case
    s = Solver(Config.from_workload(wl, precision=EDT_MIXED))
    s.set_tuning(**shape)
    V = s.invert(dev(D)).cpu().numpy()
    assert rel_l2(V, V_or) < 1e-5


def test_line_autotune(line_case):
    from paper_0905_0238_gb300 import Config, Solver, EDT_MIXED
    wl, D, V_or = line_case
    s = Solver(Config.from_workload(wl, precision=EDT_MIXED))
    Dd = dev(D)
    V0 = s.invert(Dd).cpu().numpy()
    t = s.autotune(Dd, reps=1)
    assert t["band_budget_mb"] in (16, 32, 48, 96) and t["band_cols"] in (4, 8, 16)
    assert t["refine_shape"] in (0, 1, 2, 3) and t["invert_ms"] > 0
    V1 = s.invert(Dd).cpu().numpy()
    assert rel_l2(V1, V0) < 1e-6
    assert rel_l2(V1, V_or) < 1e-5


def test_window_ztiles_and_autotune():
    from paper_0905_0238_gb300 import Config, Solver
    tops, vel = synth.layers_gradient_staircase(1500.0, 3000.0, 130.0, 10.0, sub=2)
    wl = synth.Workload3D("t", nx=32, ny=32, dx=10.0, dy=10.0, wx=4, wy=4,
                          freq_hz=synth.freqs_uniform(3, 10.0, 40.0), eps=0.15, nz=13, dz=10.0,
                          z0=0.0, layer_top=tops, layer_vel=vel, alpha=1e-4, cutoff=1.0)
    V = synth.perturbation_blobs_3d(synth.rng_for(0, 5), wl.nx, wl.ny, wl.dx, wl.dy, wl.nz,
                                    wl.dz, wl.z0, wl.layer_top, wl.layer_vel, sigma=30.0)
    D = edt3d.forward(wl, V)
    V_or, _ = edt3d.invert(wl, D)
    s = Solver(Config.from_workload(wl))
    Dd = dev(D.astype(np.complex64))
    for zt in (2, 4, 8):
        s.set_tuning(window_ztile=zt)
        Vg = s.invert(Dd).cpu().numpy()
        assert rel_l2(Vg, V_or) < 1e-5, (zt, rel_l2(Vg, V_or))
    t = s.autotune(Dd, reps=1)
    assert t["window_ztile"] in (2, 4, 8)
    assert rel_l2(s.invert(Dd).cpu().numpy(), V_or) < 1e-5
