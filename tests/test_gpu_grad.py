"""GPU misfit gradients (edt_misfit_grad) against the FP64 oracle (oracle/grad2d.py) and
against central differences of the GPU misfit itself.

* A 64-point line, 32 depths, 6 frequencies, 5 layers: J, dJ/dV and dJ/dc against the oracle
  (J and the gradients to 1e-5 relative L2: FP32 products and sums over the
  depth and lateral axes, FP64 across frequencies).
* The config-1 geometry (512 x 512, 128 frequencies 3-60 Hz, 256 depths, 20 layers) in FP32:
  J is exactly quadratic in V, so J(V + dV) - J(V - dV) = 2 <dJ/dV, dV> for any dV;
  dJ/dc_l against central differences of the GPU misfit (steps 1e-5 and, for the deeper
  layers, the configuration's 1e-3 relative); one frequency of that geometry against the
  oracle (J, dJ/dV and dJ/dc).
* The torch.autograd binding returns the same gradients through backward().
"""
import numpy as np
import pytest

import synth
from oracle import grad2d
from oracle import edt2d
from tests.gpu_helpers import rel_l2, dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def line_workload():
    tops = np.array([0.0, 60.0, 130.0, 200.0, 260.0])
    vel = np.array([1550.0, 1900.0, 2300.0, 2100.0, 2900.0])
    return synth.Workload("grad", nx=64, dx=10.0, freq_hz=synth.freqs_uniform(6, 5.0, 40.0),
                          eps=0.15, nz=32, dz=10.0, z0=0.0, layer_top=tops, layer_vel=vel,
                          alpha=1e-3, cutoff=0.0)


def model(wl, salt, amp=0.05):
    return synth.perturbation_blobs(synth.rng_for(3, salt), wl.nx, wl.dx, wl.nz, wl.dz, wl.z0,
                                    wl.layer_top, wl.layer_vel, nblob=3, sigma=25.0, amp=amp)


def solver(wl, **kw):
    from paper_0905_0238_gb300 import Config, Solver, EDT_MIXED
    return Solver(Config.from_workload(wl, precision=EDT_MIXED, **kw))


def test_misfit_gradients_match_oracle():
    wl = line_workload()
    D = edt2d.forward(wl, model(wl, 1))
    D = D + synth.noise_snr(synth.rng_for(3, 5), D, 20.0)
    V = model(wl, 2)
    J_or = grad2d.misfit(wl, V, D)
    gV_or = grad2d.grad_V(wl, V, D)
    gc_or = grad2d.grad_c(wl, V, D)
    s = solver(wl)
    J, gV, gc = s.misfit_grad(dev(V), dev(D))
    J = float(J.cpu())
    assert abs(J - J_or) < 1e-5 * J_or, (J, J_or)
    assert rel_l2(gV.cpu().numpy(), gV_or) < 1e-5, rel_l2(gV.cpu().numpy(), gV_or)
    assert rel_l2(gc.cpu().numpy(), gc_or) < 1e-5, (gc.cpu().numpy(), gc_or)
    # complex64 data and a float32 model give the same result to FP32 accuracy
    J32, gV32, gc32 = s.misfit_grad(dev(V.astype(np.float32)), dev(D.astype(np.complex64)))
    assert abs(float(J32.cpu()) - J_or) < 1e-5 * J_or
    assert rel_l2(gV32.cpu().numpy(), gV_or) < 1e-5
    assert rel_l2(gc32.cpu().numpy(), gc_or) < 1e-5


def test_autograd_binding():
    from paper_0905_0238_gb300.autograd import born_misfit
    wl = line_workload()
    D = dev(edt2d.forward(wl, model(wl, 1)))
    V = dev(model(wl, 2)).requires_grad_(True)
    vel = torch.tensor(wl.layer_vel, dtype=torch.float64, requires_grad=True)
    s = solver(wl)
    J = born_misfit(s, V, vel, D)
    (3.0 * J).backward()
    J2, gV, gc = s.misfit_grad(V.detach(), D)
    # a second call sums in another order (FP64 atomics across frequencies)
    assert abs(float(J.detach()) - float(J2)) < 1e-12 * float(J2)
    assert rel_l2(V.grad.cpu().numpy(), 3.0 * gV.cpu().numpy()) < 1e-6
    assert rel_l2(vel.grad.numpy(), 3.0 * gc.cpu().numpy()) < 1e-6


def test_config1_geometry_properties():
    wl = synth.preset("production_2d")
    wl.cutoff = 0.0
    rng = synth.rng_for(3, 11)
    Vt = synth.perturbation_random_field(rng, wl.nx, wl.dx, wl.nz, wl.dz, wl.z0, wl.layer_top,
                                         wl.layer_vel)
    s = solver(wl)
    D = s.forward(dev(Vt.astype(np.float32)), out_dtype=torch.complex64)
    D = D + dev(synth.noise_snr(rng, D.cpu().numpy(), 20.0))
    V = dev((0.5 * Vt).astype(np.float32))
    J, gV, gc = s.misfit_grad(V, D)
    J = float(J.cpu())
    assert np.isfinite(J) and J > 0
    # exact quadratic: J(V + dV) - J(V - dV) = 2 <gV, dV>
    dV = dev((0.2 * synth.perturbation_random_field(rng, wl.nx, wl.dx, wl.nz, wl.dz, wl.z0,
                                                    wl.layer_top, wl.layer_vel)).astype(np.float32))
    Jp = float(s.misfit_grad(V + dV, D)[0].cpu())
    Jm = float(s.misfit_grad(V - dV, D)[0].cpu())
    lin = 2.0 * float(torch.sum(gV.double() * dV.double()).cpu())
    assert abs((Jp - Jm) - lin) < 1e-3 * abs(lin), (Jp - Jm, lin)
    # dJ/dc_l against central differences of the GPU misfit.  The configuration's step of
    # 1e-3 relative is inside the linear regime for the deeper layers only: near-critical
    # wavenumbers (small vertical wavenumber kappa, d kappa/dc = -omega~^2/(c^3 kappa)) make J
    # strongly curved in the shallow-layer velocities at that scale, so those are checked
    # with a step of 1e-5 (the differences converge onto the gradient as the step shrinks).
    vel0 = wl.layer_vel.copy()
    scale = float(torch.max(torch.abs(gc)).cpu())

    def fd(l, rel):
        h = rel * vel0[l]
        vp, vm = vel0.copy(), vel0.copy()
        vp[l] += h
        vm[l] -= h
        s.set_reference(vp)
        Jp = float(s.misfit_grad(V, D)[0].cpu())
        s.set_reference(vm)
        Jm = float(s.misfit_grad(V, D)[0].cpu())
        s.set_reference(vel0)
        return (Jp - Jm) / (2 * h)

    for l in (0, 1, 7, 19):
        g = float(gc[l].cpu())
        d5 = fd(l, 1e-5)
        assert abs(d5 - g) < 1e-2 * max(abs(g), 1e-2 * scale), (l, d5, g)
    for l in (7, 19):
        g = float(gc[l].cpu())
        d3 = fd(l, 1e-3)
        assert abs(d3 - g) < 0.15 * max(abs(g), 1e-2 * scale), (l, d3, g)


@pytest.mark.parametrize("fi", [127, 40])
def test_config1_geometry_single_frequency_matches_oracle(fi):
    """One frequency of the config-1 geometry (512 x 512, 256 depths, 20 layers): J and
    dJ/dc against the oracle (the gradients are sums over frequencies, so one frequency is
    a sample of the full sum the oracle computes in seconds)."""
    wl = synth.preset("production_2d")
    wl.cutoff = 0.0
    wl.freq_hz = wl.freq_hz[[fi]]
    rng = synth.rng_for(3, 11)
    Vt = synth.perturbation_random_field(rng, wl.nx, wl.dx, wl.nz, wl.dz, wl.z0, wl.layer_top,
                                         wl.layer_vel)
    D = edt2d.forward(wl, Vt)
    V = 0.5 * Vt
    J_or = grad2d.misfit(wl, V, D)
    gc_or = grad2d.grad_c(wl, V, D)
    gV_or = grad2d.grad_V(wl, V, D)
    J, gV, gc = solver(wl).misfit_grad(dev(V), dev(D))
    assert abs(float(J.cpu()) - J_or) < 1e-5 * J_or
    assert rel_l2(gc.cpu().numpy(), gc_or) < 1e-5
    assert rel_l2(gV.cpu().numpy(), gV_or) < 1e-5


@pytest.mark.parametrize("fold", [1, 0])
def test_invert_adjoint_matches_oracle(fold):
    """Dbar = S^T Vbar of the mixed inversion against the oracle's adjoint (FP64 solves with
    the FP64 normal matrix): relative L2 within the mixed path's accuracy; and the
    dot-product identity <S D, Vbar> = Re <D, S^T Vbar> of the GPU pair itself."""
    from tests.gpu_helpers import small_workload
    wl = small_workload(nx=64, nz=24, nf=6, alpha=1e-3, cutoff=1.0)
    rng = np.random.default_rng(4)
    Vbar = rng.standard_normal((wl.nx, wl.nz))
    D = rng.standard_normal((6, wl.nx, wl.nx)) + 1j * rng.standard_normal((6, wl.nx, wl.nx))
    want = edt2d.invert_adjoint(wl, Vbar)
    s = solver(wl, fold=fold)
    V = s.invert(dev(D))
    Dbar = s.invert_adjoint(dev(Vbar))
    got = Dbar.cpu().numpy()
    assert rel_l2(got, want) < 1e-5, rel_l2(got, want)
    lhs = float(torch.sum(V * dev(Vbar)).cpu())
    rhs = float(np.real(np.vdot(D, got)))
    assert abs(lhs - rhs) < 1e-4 * abs(lhs), (lhs, rhs)
    # autograd: V = invert(D) and dL/dD for L = <V, Vbar>
    from paper_0905_0238_gb300.autograd import invert
    Dt = dev(D).requires_grad_(True)
    Vt = invert(s, Dt)
    torch.sum(Vt * dev(Vbar)).backward()
    assert rel_l2(Dt.grad.cpu().numpy(), got) < 1e-6


def _inv_problem(wl, salt):
    rng = synth.rng_for(7, salt)
    V = synth.perturbation_blobs(rng, wl.nx, wl.dx, wl.nz, wl.dz, wl.z0, wl.layer_top,
                                 wl.layer_vel, nblob=3, sigma=30.0, amp=0.05)
    D = edt2d.forward(wl, V)
    D = D + synth.noise_snr(synth.rng_for(7, salt + 50), D, 20.0)
    Vbar = rng.standard_normal((wl.nx, wl.nz))
    return D, Vbar


@pytest.mark.parametrize("fold,alpha", [(1, 1e-2), (0, 1e-3), (1, 1e-4)])
def test_invert_grad_c_matches_oracle(fold, alpha):
    """dL/dc_l through the damped solve for L = <V, Vbar>: the GPU's reverse mode (row
    cotangents gathered per table row, the depth march reversed) against the oracle's forward
    mode (the derivative of the normal equations, lam included, one layer at a time); a second
    call gives the same bits (the forward's data and factors are kept)."""
    from tests.gpu_helpers import small_workload
    wl = small_workload(nx=64, nz=24, nf=6, alpha=alpha, cutoff=1.0)
    D, Vbar = _inv_problem(wl, 20 + fold)
    gc_or = grad2d.invert_grad_c(wl, D, Vbar)
    s = solver(wl, fold=fold, refine=2 if alpha < 1e-3 else 1)
    s.invert(dev(D))
    Dbar, gc = s.invert_vjp(dev(Vbar))
    g = gc.cpu().numpy()
    assert rel_l2(g, gc_or) < 1e-5, rel_l2(g, gc_or)
    Dbar2, gc2 = s.invert_vjp(dev(Vbar))
    assert np.array_equal(gc2.cpu().numpy(), g)
    # Dbar alone, as edt_invert_adjoint gives it
    assert rel_l2(Dbar.cpu().numpy(), s.invert_adjoint(dev(Vbar)).cpu().numpy()) < 1e-6


def test_invert_autograd_returns_the_layer_gradient():
    from tests.gpu_helpers import small_workload
    from paper_0905_0238_gb300.autograd import invert
    wl = small_workload(nx=64, nz=24, nf=6, alpha=1e-2, cutoff=1.0)
    D, Vbar = _inv_problem(wl, 31)
    s = solver(wl)
    Dt = dev(D).requires_grad_(True)
    vel = torch.tensor(wl.layer_vel, dtype=torch.float64, requires_grad=True)
    V = invert(s, Dt, layer_vel=vel)
    torch.sum(V * dev(Vbar)).backward()
    gc_or = grad2d.invert_grad_c(wl, D, Vbar)
    assert vel.grad is not None and vel.grad.shape == (len(wl.layer_vel),)
    assert rel_l2(vel.grad.numpy(), gc_or) < 1e-5
    assert rel_l2(Dt.grad.cpu().numpy(), edt2d.invert_adjoint(wl, Vbar)) < 1e-5


def test_invert_grad_c_production_geometry_single_frequency():
    """One frequency of the 512 x 512, 256-depth, 20-layer line with the evanescent cut: dL/dc
    of three layers against the oracle (one frequency keeps the oracle's solves to seconds)."""
    wl = synth.preset("production_2d")
    wl.freq_hz = wl.freq_hz[[60]]
    D, Vbar = _inv_problem(wl, 40)
    s = solver(wl)
    s.invert(dev(D))
    _, gc = s.invert_vjp(dev(Vbar), want_D=False)
    g = gc.cpu().numpy()
    layers = [0, 7, 19]
    want = np.array([float(np.sum(Vbar * grad2d.invert_tangent(wl, D, l)[1])) for l in layers])
    assert rel_l2(g[layers], want) < 1e-5, (g[layers], want)
