"""Edge cases of the GPU paths against the oracle: the largest lateral size (1024), a single
depth, a single frequency, a homogeneous (one-layer) reference, and gradients at a depth
count that is not a multiple of the kernels' depth tiles."""
import numpy as np
import pytest

import synth
from oracle import edt2d, grad2d
from tests.gpu_helpers import rel_l2, small_workload, blobs, dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def mixed(wl, **kw):
    from paper_0905_0238_gb300 import Config, Solver, EDT_MIXED
    return Solver(Config.from_workload(wl, precision=EDT_MIXED, **kw))


def data(wl, salt):
    D = edt2d.forward(wl, blobs(wl, salt=salt))
    return D + synth.noise_snr(synth.rng_for(5, salt), D, 20.0)


@pytest.mark.parametrize("case", ["nx1024", "nz1", "nf1", "one_layer"])
def test_invert_edge_cases_match_oracle(case):
    if case == "nx1024":
        wl = small_workload(nx=1024, nz=16, nf=2, dx=5.0, alpha=1e-3)
    elif case == "nz1":
        wl = small_workload(nx=64, nz=1, nf=6, alpha=1e-3)
    elif case == "nf1":
        wl = small_workload(nx=64, nz=24, nf=1, fmin=20.0, fmax=20.0, alpha=1e-3)
    else:
        wl = small_workload(nx=64, nz=24, nf=6, alpha=1e-3,
                            layers=(np.array([0.0]), np.array([2000.0])))
    D = data(wl, 3)
    V_or, vh_or = edt2d.invert(wl, D)
    s = mixed(wl)
    V = s.invert(dev(D.astype(np.complex64))).cpu().numpy()
    st = s.stats()
    assert st.n_notpd == 0 and st.n_nonfinite == 0
    assert rel_l2(s.vhat().cpu().numpy(), vh_or) < 1e-5
    assert rel_l2(V, V_or) < 1e-5


@pytest.mark.parametrize("case", ["nz37_nx128", "one_layer"])
def test_misfit_gradient_edge_cases_match_oracle(case):
    if case == "nz37_nx128":
        tops = np.array([0.0, 90.0, 200.0])
        vel = np.array([1600.0, 2200.0, 2700.0])
        wl = synth.Workload("g", nx=128, dx=10.0, freq_hz=synth.freqs_uniform(3, 8.0, 30.0),
                            eps=0.15, nz=37, dz=10.0, z0=5.0, layer_top=tops, layer_vel=vel,
                            alpha=1e-3, cutoff=0.0)
    else:
        wl = synth.Workload("g", nx=64, dx=10.0, freq_hz=synth.freqs_uniform(4, 8.0, 30.0),
                            eps=0.15, nz=20, dz=10.0, z0=0.0, layer_top=np.array([0.0]),
                            layer_vel=np.array([2000.0]), alpha=1e-3, cutoff=0.0)
    D = data(wl, 4)
    V = blobs(wl, salt=6)
    J_or = grad2d.misfit(wl, V, D)
    gV_or = grad2d.grad_V(wl, V, D)
    gc_or = grad2d.grad_c(wl, V, D)
    J, gV, gc = mixed(wl).misfit_grad(dev(V), dev(D))
    assert abs(float(J.cpu()) - J_or) < 1e-5 * J_or
    assert rel_l2(gV.cpu().numpy(), gV_or) < 1e-4
    assert rel_l2(gc.cpu().numpy(), gc_or) < 1e-4
