"""The adjoint Born operator edt_adjoint (V = F^T D) against the oracle's adjoint and by the
dot-product identity with edt_forward.

FP64 path 1e-10 against oracle.edt2d.adjoint; mixed path 1e-5 (FP32 transform and table);
<F V, D> = <V, F^T D> on seeded random V and D at test sizes and on the production geometry
(512 x 512, 128 frequencies, 256 depths), a property that holds at any size, to a fraction of
the Cauchy-Schwarz scale ||F V|| ||D|| (both sides are cancelling sums of random terms).
"""
import numpy as np
import pytest

import synth
from oracle import edt2d
from tests.gpu_helpers import rel_l2, small_workload, dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


LAYERS = (np.array([0.0, 60.0, 150.0, 250.0]), np.array([1500.0, 1800.0, 2300.0, 2900.0]))


def _solver(wl, precision):
    from paper_0905_0238_gb300 import Config, Solver
    return Solver(Config.from_workload(wl, precision=precision))


def _random_data(wl, salt, dtype=np.complex128):
    return synth.random_data(synth.rng_for(6, salt=salt), (len(wl.freq_hz), wl.nx, wl.nx), dtype)


@pytest.mark.parametrize("nx,nz,nf", [(32, 24, 5), (64, 37, 4)])
def test_adjoint_fp64_matches_oracle(nx, nz, nf):
    from paper_0905_0238_gb300 import EDT_FP64
    wl = small_workload(nx=nx, nz=nz, nf=nf)
    D = _random_data(wl, salt=nx + nz)
    want = edt2d.adjoint(wl, D)
    got = _solver(wl, EDT_FP64).adjoint(dev(D)).cpu().numpy()
    assert rel_l2(got, want) < 1e-10


@pytest.mark.parametrize("nx,nz,nf", [(64, 32, 5), (128, 45, 3)])
def test_adjoint_mixed_matches_oracle(nx, nz, nf):
    from paper_0905_0238_gb300 import EDT_MIXED
    wl = small_workload(nx=nx, nz=nz, nf=nf, alpha=1e-2, layers=LAYERS)
    D = _random_data(wl, salt=nx + nz + 1, dtype=np.complex64)
    want = edt2d.adjoint(wl, D.astype(np.complex128))
    got = _solver(wl, EDT_MIXED).adjoint(dev(D), out_dtype=torch.float32).cpu().numpy()
    assert rel_l2(got, want) < 1e-5


def _dot_identity(s, wl, salt, ddtype):
    rng = synth.rng_for(6, salt=salt)
    V = torch.from_numpy(rng.standard_normal((wl.nx, wl.nz))).cuda()
    D = torch.from_numpy(np.ascontiguousarray(_random_data(wl, salt + 1, ddtype))).cuda()
    FV = s.forward(V, out_dtype=torch.complex128)
    FtD = s.adjoint(D)
    lhs = float(torch.sum(FV.real * D.real.double() + FV.imag * D.imag.double()))
    rhs = float(torch.sum(V * FtD))
    # random V and D make both sides cancelling sums; the Cauchy-Schwarz bound sets the scale
    scale = float(torch.linalg.norm(FV)) * float(torch.linalg.norm(D.to(torch.complex128)))
    return lhs, rhs, scale


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-6)])
def test_adjoint_dot_product_identity(precision, tol):
    wl = small_workload(nx=64, nz=30, nf=4, alpha=1e-2, layers=LAYERS)
    lhs, rhs, scale = _dot_identity(_solver(wl, precision), wl, 11, np.complex128)
    assert abs(lhs - rhs) <= tol * scale


def test_adjoint_dot_product_identity_production_geometry():
    """Mixed path on the full production geometry."""
    from paper_0905_0238_gb300 import EDT_MIXED
    wl = synth.preset("production_2d")
    s = _solver(wl, EDT_MIXED)
    lhs, rhs, scale = _dot_identity(s, wl, 21, np.complex64)
    assert abs(lhs - rhs) <= 1e-6 * scale
    # the FP64 adjoint of the same geometry on one frequency, against the mixed one
    wl1 = synth.preset("production_2d")
    wl1.freq_hz = wl1.freq_hz[[77]]
    D = dev(_random_data(wl1, 5, np.complex64))
    a64 = _solver(wl1, 0).adjoint(D.to(torch.complex128))
    a32 = _solver(wl1, EDT_MIXED).adjoint(D)
    assert rel_l2(a32.cpu().numpy(), a64.cpu().numpy()) < 1e-5
