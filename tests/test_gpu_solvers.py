"""The paper's solver variants on the GPU (FP64 line path) against the oracle: the truncated
SVD (tolerance relative and absolute, odd and even depth counts) and the vertical-wavenumber
disk with the damped solve and with the truncated SVD."""
import numpy as np
import pytest

import synth
from oracle import edt2d
from tests.gpu_helpers import rel_l2, small_workload, blobs, dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def solve_gpu(wl, D, **kw):
    from paper_0905_0238_gb300 import Config, Solver, EDT_FP64
    s = Solver(Config.from_workload(wl, precision=EDT_FP64, **kw))
    V = s.invert(dev(D)).cpu().numpy()
    st = s.stats()
    assert st.n_notpd == 0 and st.n_nonfinite == 0
    return V, s.vhat().cpu().numpy()


def separated_tol(wl, D, cands):
    """A relative tolerance no singular value of any subproblem lies within 2 % of."""
    D2 = edt2d.data_transform(D)
    ratios = []
    for m in range(wl.nx // 2 + 1):
        _, sysd = edt2d.solve_wavenumber(wl, D2, m, return_system=True)
        if "Ahat" in sysd:
            sv = np.linalg.svd(sysd["Ahat"], compute_uv=False)
            ratios.append(sv / sv[0])
    r = np.concatenate(ratios)
    for t in cands:
        if np.min(np.abs(np.log(r / t))) > 0.02:
            return t
    raise AssertionError("no separated tolerance")


def data(wl, salt):
    D = edt2d.forward(wl, blobs(wl, salt=salt))
    return D + synth.noise_snr(synth.rng_for(5, salt), D, 30.0)


@pytest.mark.parametrize("nz", [24, 33])
def test_tsvd_matches_oracle(nz):
    wl = small_workload(nx=32, nz=nz, nf=6, alpha=1e-3)
    D = data(wl, 11)
    tol = separated_tol(wl, D, [3e-3, 2e-3, 5e-3, 1.5e-3, 7e-3])
    V_or, vh_or = edt2d.invert(wl, D, solver="tsvd", tsvd_tol=-tol)
    V, vh = solve_gpu(wl, D, solver=1, tsvd_tol=-tol)
    assert rel_l2(vh, vh_or) < 1e-8 and rel_l2(V, V_or) < 1e-8


def test_tsvd_absolute_tolerance_matches_oracle():
    wl = small_workload(nx=32, nz=20, nf=6, alpha=1e-3)
    D = data(wl, 12)
    rel = separated_tol(wl, D, [1e-2, 2e-2, 5e-3])
    # an absolute sigma: the relative one times the largest singular value of subproblem 0
    D2 = edt2d.data_transform(D)
    _, sysd = edt2d.solve_wavenumber(wl, D2, 0, return_system=True)
    smax0 = np.linalg.svd(sysd["Ahat"], compute_uv=False)[0]
    sig = rel * smax0
    V_or, vh_or = edt2d.invert(wl, D, solver="tsvd", tsvd_tol=sig)
    V, vh = solve_gpu(wl, D, solver=1, tsvd_tol=sig)
    assert rel_l2(vh, vh_or) < 1e-8


@pytest.mark.parametrize("factor", [0.8, 1.5])
def test_disk_damped_matches_oracle(factor):
    wl = small_workload(nx=32, nz=40, nf=6, alpha=1e-3)
    D = data(wl, 13)
    V_or, vh_or = edt2d.invert(wl, D, kz_disk=factor)
    V, vh = solve_gpu(wl, D, kz_disk=factor)
    assert rel_l2(vh, vh_or) < 1e-10 and rel_l2(V, V_or) < 1e-10


def test_disk_tsvd_paper_shaped_matches_oracle():
    # depths of the paper's examples: 65 samples (odd: no Nyquist vector), disk factor 2.2
    wl = small_workload(nx=32, nz=65, nf=8, dz=10.0, fmin=2.0, fmax=12.0, alpha=1e-3)
    D = data(wl, 14)
    tol = 1e-3
    V_or, vh_or = edt2d.invert(wl, D, solver="tsvd", tsvd_tol=-tol, kz_disk=2.2)
    V, vh = solve_gpu(wl, D, solver=1, tsvd_tol=-tol, kz_disk=2.2)
    assert rel_l2(vh, vh_or) < 1e-8
