"""Parity at the full production size, in the launch configuration bench.py times.

The 512 x 512 x 128-frequency x 256-depth workload (20 layers, alpha = 1e-2) is inverted
on the GPU by the mixed path (split tensor-core Gram, FP64-class Cholesky, one refinement
step, reciprocal folding) and by the plain FP64 path; the FP64 oracle solves a sample of
midpoint wavenumbers (it cannot afford all 257 split systems in a test).  Sampled Vhat are
compared one by one: 1e-5 relative for the mixed path, 1e-10 for the FP64 path.  Data are
seeded complex64 values of the workload's shape (any data define a valid least-squares
problem).  Properties that hold at any size are checked on the full output: V is real by
construction, Vhat is zero for no wavenumber with rows, and the row counts match the cut.
"""
import numpy as np
import pytest

import synth
from oracle import edt2d
from tests.gpu_helpers import rel_l2, dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SAMPLE_M = (0, 1, 97, 128, 201, 256)


@pytest.fixture(scope="module")
def production():
    wl = synth.preset("production_2d")
    rng = synth.rng_for(1, salt=55)
    D = synth.random_data(rng, (len(wl.freq_hz), wl.nx, wl.nx), np.complex64)
    D2 = edt2d.data_transform(D.astype(np.complex128))
    g = edt2d.green_table(wl)
    want = {m: edt2d.solve_wavenumber(wl, D2, m, g) for m in SAMPLE_M}
    return wl, D, want


def test_mixed_path_full_size_sampled_wavenumbers(production):
    from paper_0905_0238_gb300 import Config, Solver, EDT_MIXED
    wl, D, want = production
    s = Solver(Config.from_workload(wl, precision=EDT_MIXED, passes=3, refine=1, fold=1))
    V = s.invert(dev(D), out_dtype=torch.float32)
    vh = s.vhat().cpu().numpy()
    st = s.stats()
    assert st.n_notpd == 0 and st.n_nonfinite == 0
    for m in SAMPLE_M:
        assert rel_l2(vh[m], want[m]) < 1e-5, (m, rel_l2(vh[m], want[m]))
    counts = s.row_counts()
    assert np.all(np.abs(vh[counts > 0]).max(axis=1) > 0)
    assert torch.isfinite(V).all()
    for m in (1, 128, 256):
        assert counts[m] == len(edt2d.kept_rows(wl, m))


def test_fp64_path_full_size_sampled_wavenumbers(production):
    from paper_0905_0238_gb300 import Config, Solver, EDT_FP64
    wl, D, want = production
    s = Solver(Config.from_workload(wl, precision=EDT_FP64))
    s.invert(dev(D))
    vh = s.vhat().cpu().numpy()
    for m in SAMPLE_M:
        assert rel_l2(vh[m], want[m]) < 1e-10, (m, rel_l2(vh[m], want[m]))
