"""GPU parity where the data transform runs in several chunks of frequency planes.

With freq_chunk = 16 the spectrum buffer holds 16 planes at a time, so a 512-wide
workload with 41 frequencies runs the transform, the right-hand-side gather and the
forward model in 3 chunks with a ragged last chunk; the automatic size (256 MB of
planes) takes all 41 in one.  Compared with the FP64 oracle: the forward model to
1e-11 (FP64) and 1e-5 (FP32 spectrum), the inversion to 1e-10 (FP64) and 1e-5 (mixed).
"""
import numpy as np
import pytest

import synth
from oracle import edt2d
from tests.gpu_helpers import rel_l2, small_workload, blobs, dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NX, NZ, NF = 512, 12, 41


@pytest.fixture(scope="module")
def case():
    wl = small_workload(nx=NX, nz=NZ, nf=NF, dx=12.5, dz=8.0, fmin=3.0, fmax=60.0, alpha=1e-3)
    V = blobs(wl, salt=3)
    g = edt2d.green_table(wl)
    D = edt2d.forward(wl, V, g=g)
    D = D + synth.noise_snr(synth.rng_for(0, salt=77), D, 20.0)
    V_or, vh_or = edt2d.invert(wl, D)
    return wl, V, D, V_or, vh_or


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_forward_spans_chunks(case, precision):
    from paper_0905_0238_gb300 import Config, Solver, EDT_FP64, EDT_MIXED
    wl, V, _, _, _ = case
    prec = EDT_FP64 if precision == "fp64" else EDT_MIXED
    s = Solver(Config.from_workload(wl, precision=prec, freq_chunk=16))
    assert s.stats().freq_chunk == 16
    want = edt2d.forward(wl, V)
    D = s.forward(torch.from_numpy(V).cuda()).cpu().numpy()
    assert rel_l2(D, want) < (1e-11 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_invert_spans_chunks(case, precision):
    from paper_0905_0238_gb300 import Config, Solver, EDT_FP64, EDT_MIXED
    wl, _, D, V_or, vh_or = case
    prec = EDT_FP64 if precision == "fp64" else EDT_MIXED
    s = Solver(Config.from_workload(wl, precision=prec, freq_chunk=16))
    st = s.stats()
    nchunk = -(-NF // st.freq_chunk)
    assert nchunk >= 3 and NF % st.freq_chunk != 0
    D_in = D if precision == "fp64" else D.astype(np.complex64)
    V_gpu = s.invert(dev(D_in)).cpu().numpy()
    tol = 1e-10 if precision == "fp64" else 1e-5
    assert rel_l2(s.vhat().cpu().numpy(), vh_or) < tol
    assert rel_l2(V_gpu, V_or) < tol


def test_automatic_chunk_takes_every_plane_that_fits(case):
    from paper_0905_0238_gb300 import Config, Solver, EDT_FP64
    wl = case[0]
    assert Solver(Config.from_workload(wl, precision=EDT_FP64)).stats().freq_chunk == NF
