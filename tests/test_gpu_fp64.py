"""GPU parity of the plain-FP64 path against the FP64 oracle (through the C ABI).

Stages: depth march (g), spectral Born forward model, and the whole inversion
(transform, split right-hand sides, FP64 normal matrices, FP64 Cholesky, inverse
transform).  Tolerances: g to 1e-12, forward to 1e-11, V and Vhat to 1e-10 relative L2
(the systems here satisfy cond(G + lam I) * 2^-53 < 1e-11).
"""
import numpy as np
import pytest

import synth
from oracle import edt2d
from tests.gpu_helpers import rel_l2, small_workload, blobs, dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def solver(wl, **kw):
    from paper_0905_0238_gb300 import Config, Solver, EDT_FP64
    return Solver(Config.from_workload(wl, precision=EDT_FP64, **kw))


@pytest.mark.parametrize("nz,nlayer_sub", [(24, 2), (50, 1), (64, 4)])
def test_green_table_matches_oracle(nz, nlayer_sub):
    wl = small_workload(nx=32, nz=nz, nf=5, layers=synth.layers_gradient_staircase(
        1500.0, 3000.0, nz * 10.0, 10.0, sub=nlayer_sub))
    g = solver(wl).green().cpu().numpy()
    want = edt2d.green_table(wl)[:, : wl.nx // 2 + 1, :]
    assert rel_l2(g, want) < 1e-12
    assert np.max(np.abs(g - want) / np.abs(want)) < 1e-10


def test_green_table_production_layers():
    wl = synth.preset("production_2d")
    wl.freq_hz = wl.freq_hz[::16]
    g = solver(wl).green().cpu().numpy()
    want = edt2d.green_table(wl)[:, : wl.nx // 2 + 1, :]
    assert rel_l2(g, want) < 1e-12


@pytest.mark.parametrize("nx,nz", [(16, 8), (32, 24), (64, 40)])
def test_forward_matches_oracle(nx, nz):
    wl = small_workload(nx=nx, nz=nz, nf=4)
    V = blobs(wl, salt=1)
    s = solver(wl)
    D = s.forward(torch.from_numpy(V).cuda()).cpu().numpy()
    want = edt2d.forward(wl, V)
    assert rel_l2(D, want) < 1e-11


@pytest.mark.parametrize("fold", [0, 1])
def test_invert_small_2d_matches_oracle(fold):
    """The 64 x 64 x 32-frequency x 64-depth FP64 workload, Born data, noise free."""
    wl = synth.preset("small_2d")
    V = synth.perturbation_blobs(synth.rng_for(0), wl.nx, wl.dx, wl.nz, wl.dz, wl.z0,
                                 wl.layer_top, wl.layer_vel)
    D = edt2d.forward(wl, V)
    V_or, vh_or = edt2d.invert(wl, D)
    s = solver(wl, fold=fold)
    V_gpu = s.invert(dev(D)).cpu().numpy()
    vh_gpu = s.vhat().cpu().numpy()
    st = s.stats()
    assert st.n_notpd == 0 and st.n_nonfinite == 0
    assert rel_l2(vh_gpu, vh_or) < 1e-10
    assert rel_l2(V_gpu, V_or) < 1e-10


@pytest.mark.parametrize("nx,nz,nf,cutoff", [(32, 50, 5, 1.0), (16, 7, 3, 0.0), (64, 130, 4, 1.0)])
def test_invert_ragged_matches_oracle(nx, nz, nf, cutoff):
    """Depth counts that are not tile multiples, the cut on and off, noisy data."""
    wl = small_workload(nx=nx, nz=nz, nf=nf, alpha=1e-3, cutoff=cutoff)
    rng = synth.rng_for(0, salt=5)
    D = synth.random_data(rng, (nf, nx, nx))
    V_or, vh_or = edt2d.invert(wl, D)
    s = solver(wl)
    V_gpu = s.invert(dev(D)).cpu().numpy()
    assert rel_l2(s.vhat().cpu().numpy(), vh_or) < 1e-10
    assert rel_l2(V_gpu, V_or) < 1e-10


def test_invert_complex64_input_and_float32_output():
    wl = small_workload(nx=32, nz=20, nf=4, alpha=1e-3)
    D = synth.random_data(synth.rng_for(0, salt=6), (4, 32, 32), np.complex64)
    V_or, _ = edt2d.invert(wl, D.astype(np.complex128))
    s = solver(wl)
    V32 = s.invert(dev(D), out_dtype=torch.float32).cpu().numpy()
    assert V32.dtype == np.float32
    assert rel_l2(V32, V_or) < 1e-6


def test_invert_host_buffers():
    wl = small_workload(nx=32, nz=20, nf=4, alpha=1e-3)
    D = synth.random_data(synth.rng_for(0, salt=7), (4, 32, 32))
    V_or, _ = edt2d.invert(wl, D)
    s = solver(wl)
    Dh = torch.from_numpy(D).pin_memory()
    Vh = torch.empty((32, 20), dtype=torch.float64).pin_memory()
    s.invert_host(Dh, Vh)
    torch.cuda.synchronize()
    assert rel_l2(Vh.numpy(), V_or) < 1e-10


def test_empty_subproblems_are_zero():
    """A cut that removes every row of some wavenumbers leaves those Vhat exactly zero."""
    wl = small_workload(nx=64, nz=16, nf=2, fmin=5.0, fmax=8.0, dx=5.0, alpha=1e-3)
    counts = None
    s = solver(wl)
    counts = s.row_counts()
    assert (counts == 0).any()
    D = synth.random_data(synth.rng_for(0, salt=8), (2, 64, 64))
    _, vh_or = edt2d.invert(wl, D)
    s.invert(dev(D))
    vh = s.vhat().cpu().numpy()
    assert np.all(vh[counts == 0] == 0)
    assert rel_l2(vh, vh_or) < 1e-10
