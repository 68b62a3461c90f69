"""GPU parity of the mixed-precision path (tcgen05 Gram + FP64-class Cholesky + refinement).

The tensor-core normal matrices are compared with Ahat^T Ahat formed in FP64 from the
oracle's own kernel rows (a matmul in the test; the oracle itself never forms a Gram);
the end-to-end inversion with the oracle's QR solution.  Tolerances: Gram relative
Frobenius 5e-3 with one 16-bit operand pass, 2e-5 with the split hi/lo operands; trace(G)
5e-7 (the FP32 table sqrt|s_f| g is accurate to ~2e-7 relative: FP64-reduced arguments, FP32
sincos/exp2, so each |a|^2 carries up to ~5e-7);
V and Vhat 1e-5 relative L2 after one refinement step, and at weak damping (alpha down to
1e-6, the FP64-accurate residual, one to three steps) on noisy data.
"""
import numpy as np
import pytest

import synth
from oracle import edt2d
from tests.gpu_helpers import rel_l2, small_workload, blobs, dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def solver(wl, passes=3, refine=1, fold=1):
    from paper_0905_0238_gb300 import Config, Solver, EDT_MIXED
    return Solver(Config.from_workload(wl, precision=EDT_MIXED, passes=passes, refine=refine,
                                       fold=fold))


def born_data(wl, salt=0, snr_db=20.0):
    V = blobs(wl, salt=salt)
    D = edt2d.forward(wl, V)
    if snr_db is not None:
        D = D + synth.noise_snr(synth.rng_for(0, salt=salt + 100), D, snr_db)
    return np.ascontiguousarray(D.astype(np.complex64))


@pytest.mark.parametrize("passes", [1, 3])
@pytest.mark.parametrize("nz", [40, 130, 256])
def test_gram_tc_matches_fp64_normal_matrix(passes, nz):
    wl = small_workload(nx=32, nz=nz, nf=4, alpha=1e-2, dz=8.0)
    D = born_data(wl, salt=1)
    G, b, tr = solver(wl, passes=passes).gram(dev(D))
    G, b, tr = G.cpu().numpy(), b.cpu().numpy(), tr.cpu().numpy()
    D2 = edt2d.data_transform(D.astype(np.complex128))
    tolG = 5e-3 if passes == 1 else 2e-5
    for m in range(wl.nx // 2 + 1):
        _, sysd = edt2d.solve_wavenumber(wl, D2, m, return_system=True)
        if len(sysd["rows"]) == 0:
            assert np.all(G[m] == 0) and tr[m] == 0
            continue
        Ah, dh = sysd["Ahat"], sysd["dhat"]
        Gr = Ah.T @ Ah
        br = Ah.T @ dh
        assert rel_l2(G[m], Gr) < tolG, (m, rel_l2(G[m], Gr))
        assert rel_l2(b[m][:, : br.shape[1]], br) < 5 * tolG
        assert abs(tr[m] - np.trace(Gr)) <= 5e-7 * np.trace(Gr)


@pytest.mark.parametrize("passes,refine", [(3, 1), (1, 2)])
@pytest.mark.parametrize("nx,nz,nf", [(32, 40, 6), (32, 41, 5), (64, 130, 4), (32, 256, 3)])
def test_invert_mixed_matches_oracle(passes, refine, nx, nz, nf):
    """Split BF16x3 Gram + one refinement step (or BF16 Gram + two steps) reach 1e-5."""
    wl = small_workload(nx=nx, nz=nz, nf=nf, alpha=1e-2, dz=8.0)
    D = born_data(wl, salt=2)
    V_or, vh_or = edt2d.invert(wl, D.astype(np.complex128))
    s = solver(wl, passes=passes, refine=refine)
    V = s.invert(dev(D)).cpu().numpy()
    vh = s.vhat().cpu().numpy()
    st = s.stats()
    assert st.n_notpd == 0 and st.n_nonfinite == 0
    assert rel_l2(vh, vh_or) < 1e-5
    assert rel_l2(V, V_or) < 1e-5


def test_refinement_is_what_reaches_the_tolerance():
    """Without refinement the BF16 Gram leaves a visible error; one step removes it."""
    wl = small_workload(nx=32, nz=64, nf=6, alpha=1e-2, dz=8.0)
    D = born_data(wl, salt=3)
    V_or, _ = edt2d.invert(wl, D.astype(np.complex128))
    e0 = rel_l2(solver(wl, passes=1, refine=0).invert(dev(D)).cpu().numpy(), V_or)
    e1 = rel_l2(solver(wl, passes=1, refine=1).invert(dev(D)).cpu().numpy(), V_or)
    e2 = rel_l2(solver(wl, passes=1, refine=2).invert(dev(D)).cpu().numpy(), V_or)
    assert e0 > 1e-5
    assert e1 < e0 / 10 and e2 <= e1 * 1.01 + 1e-9


def test_mixed_without_folding_and_without_cut():
    wl = small_workload(nx=32, nz=48, nf=4, alpha=1e-2, cutoff=0.0, dz=8.0)
    D = born_data(wl, salt=4)
    V_or, _ = edt2d.invert(wl, D.astype(np.complex128))
    for fold in (0, 1):
        V = solver(wl, fold=fold).invert(dev(D)).cpu().numpy()
        assert rel_l2(V, V_or) < 1e-5


def test_graph_replay_matches_direct_calls():
    """edt_invert captured into a CUDA graph gives the direct call's result, replayed and
    re-captured when the output buffer changes."""
    wl = small_workload(nx=32, nz=40, nf=4, alpha=1e-2, dz=8.0)
    D = born_data(wl, salt=6)
    s = solver(wl)
    ref = s.invert(dev(D)).cpu().numpy()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s.set_graph(True)
        Dd = dev(D)
        out1 = torch.empty((wl.nx, wl.nz), device="cuda", dtype=torch.float64)
        out2 = torch.empty_like(out1)
        for out in (out1, out1, out1, out2, out2):
            out.fill_(float("nan"))
            s.invert(Dd, out=out)
            st.synchronize()
            # every cross-block sum runs in a fixed order: the same bits as the direct call
            assert np.array_equal(out.cpu().numpy(), ref)
        s.set_graph(False)


@pytest.mark.parametrize("nx,nz,nf,alpha", [(32, 40, 6, 1e-2), (64, 130, 4, 1e-2), (32, 256, 3, 1e-2),
                                             (32, 256, 3, 1e-5), (64, 33, 5, 1e-4)])
def test_double_float_cholesky_matches_native_fp64(nx, nz, nf, alpha):
    """The double-float factorisation (the mixed path's default: FP32 pairs with error-free
    products and sums, FP64 pivots) gives the native-FP64 factor of the same normal matrix
    to 1e-13 relative per subproblem at alpha = 1e-2, and the same refined solution.  At
    weaker damping both factors' sensitivity grows with kappa = cond(G + lam I) (the FP64
    factor itself carries ~kappa 2^-53), so there the bound is max(1e-13, 8 kappa 2^-48): the
    double-float unit roundoff scaled by the conditioning, with a small constant for the
    rounding accumulated over the n operations of each entry; kappa is estimated from the
    pivots, (max L_ii / min L_ii)^2."""
    from paper_0905_0238_gb300 import Config, Solver, EDT_MIXED
    wl = small_workload(nx=nx, nz=nz, nf=nf, alpha=alpha, dz=8.0)
    D = born_data(wl, salt=7)
    V_or, _ = edt2d.invert(wl, D.astype(np.complex128))
    out = {}
    for mode in (1, 2):
        s = Solver(Config.from_workload(wl, precision=EDT_MIXED, passes=3, refine=1, chol_df=mode))
        V = s.invert(dev(D)).cpu().numpy()
        assert s.stats().n_notpd == 0
        out[mode] = (V, np.tril(s.factor().cpu().numpy()))
    (Vdf, Ldf), (V64, L64) = out[1], out[2]
    for m in range(Ldf.shape[0]):
        if np.any(L64[m]):
            dg = np.abs(np.diag(L64[m]))
            kappa = (dg.max() / dg.min()) ** 2
            tol = 1e-13 if alpha >= 1e-2 else max(1e-13, 8 * kappa * 2.0 ** -48)
            assert rel_l2(Ldf[m], L64[m]) < tol, (m, rel_l2(Ldf[m], L64[m]), kappa)
    # after one refinement step the solution still depends, at first order, on the FP32 copy
    # of the factor used by the correction solve, whose last bits differ between the two
    # factorisations; at weak damping the conditioning amplifies that (both stay ~1e-6 from
    # the oracle)
    assert rel_l2(Vdf, V64) < (1e-10 if alpha >= 1e-2 else 1e-7)
    assert rel_l2(Vdf, V_or) < 1e-5 and rel_l2(V64, V_or) < 1e-5


def _noisy_case(case, alpha):
    import synth as _s
    if case == "prod_layers":
        wp = _s.preset("production_2d")
        return small_workload(nx=64, nz=128, nf=8, alpha=alpha, dz=8.0, layers=(wp.layer_top, wp.layer_vel))
    nx, nz, nf = {"grad40": (32, 40, 6), "grad130": (64, 130, 4), "grad256": (32, 256, 3)}[case]
    return small_workload(nx=nx, nz=nz, nf=nf, alpha=alpha, dz=8.0)


@pytest.mark.parametrize("alpha,refine", [(1e-4, 1), (1e-5, 1), (1e-6, 3)])
@pytest.mark.parametrize("case", ["grad40", "grad130", "grad256", "prod_layers"])
def test_invert_mixed_weak_damping(case, alpha, refine):
    """Weak damping on 20 dB data: the split FP16 Gram sets the refinement's contraction and
    the FP64-accurate residual (chosen automatically below alpha = 1e-3) its limit; one step
    reaches 1e-5 down to alpha = 1e-5, three steps at 1e-6."""
    wl = _noisy_case(case, alpha)
    D = born_data(wl, salt=2)
    V_or, vh_or = edt2d.invert(wl, D.astype(np.complex128))
    s = solver(wl, passes=3, refine=refine)
    V = s.invert(dev(D)).cpu().numpy()
    st = s.stats()
    assert st.n_notpd == 0 and st.n_nonfinite == 0
    assert rel_l2(s.vhat().cpu().numpy(), vh_or) < 1e-5
    assert rel_l2(V, V_or) < 1e-5, rel_l2(V, V_or)


def test_fp64_accurate_residual_lowers_the_weak_damping_floor():
    """At alpha = 1e-6 with three steps, the FP32 residual (FP32 table and products) stalls
    above the double-float residual's error."""
    from paper_0905_0238_gb300 import Config, Solver, EDT_MIXED
    wl = _noisy_case("grad40", 1e-6)
    D = born_data(wl, salt=2)
    V_or, _ = edt2d.invert(wl, D.astype(np.complex128))
    err = {}
    for resid in (1, 2):
        cfg = Config.from_workload(wl, precision=EDT_MIXED, passes=3, refine=3, resid=resid)
        err[resid] = rel_l2(Solver(cfg).invert(dev(D)).cpu().numpy(), V_or)
    assert err[2] < 1e-5 and err[2] < err[1] / 2, err


def test_shorter_gram_segments_reduce_the_accumulation_error():
    """Long FP32 tensor-memory accumulations lose low bits systematically (the diagonal is
    biased low); flushing every 32 rows to an FP64-summed partial tile shrinks the Gram's
    error against A^T A (256-point line, 128 frequencies: ~2.6 k rows per CTA segment)."""
    from paper_0905_0238_gb300 import Config, Solver, EDT_MIXED
    wp = synth.preset("production_2d")
    wl = small_workload(nx=256, nz=64, nf=128, fmin=3.0, fmax=60.0, dx=12.5, dz=8.0, alpha=1e-2,
                        layers=(wp.layer_top, wp.layer_vel))
    D = synth.random_data(synth.rng_for(3, salt=77), (len(wl.freq_hz), wl.nx, wl.nx), np.complex64)
    D2 = edt2d.data_transform(D.astype(np.complex128))
    g = edt2d.green_table(wl)
    refs = {}
    for m in (0, 20, 120):
        _, sysd = edt2d.solve_wavenumber(wl, D2, m, g=g, return_system=True)
        refs[m] = sysd["Ahat"].T @ sysd["Ahat"]
    err = {}
    for cap in (0, 32):
        s = Solver(Config.from_workload(wl, precision=EDT_MIXED, passes=3, gram_seg_rows=cap))
        G = s.gram(dev(D))[0].cpu().numpy()
        err[cap] = max(rel_l2(G[m], refs[m]) for m in refs)
    assert err[32] < err[0] / 3 and err[32] < 5e-6, err


@pytest.mark.parametrize("nlayer", [1, 5, 32])
def test_few_layer_reference_with_fp32_march_coefficients(nlayer):
    """A line reference of at most 32 layers with the FP32 residual (alpha >= 1e-3): the depth
    march's coefficients are formed in FP32 (kappa refined by one Newton step on the FP64
    residual, double-float phases, FP32 recursions), a few FP32 ulps per layer in the table.
    The inversion meets the oracle's 1e-5 and stays within 2e-6 of the FP64 GPU path, whose
    table comes from the FP64 march."""
    from paper_0905_0238_gb300 import Config, Solver, EDT_FP64
    nz, dz = 48, 8.0
    tops = np.linspace(0.0, nz * dz, nlayer, endpoint=False)
    vel = np.linspace(1500.0, 3000.0, nlayer)
    wl = small_workload(nx=32, nz=nz, nf=6, alpha=1e-2, dz=dz, layers=(tops, vel))
    D = born_data(wl, salt=8)
    V_or, vh_or = edt2d.invert(wl, D.astype(np.complex128))
    s = solver(wl)
    V = s.invert(dev(D)).cpu().numpy()
    vh = s.vhat().cpu().numpy()
    V64 = Solver(Config.from_workload(wl, precision=EDT_FP64)).invert(dev(D.astype(np.complex128))).cpu().numpy()
    assert rel_l2(vh, vh_or) < 1e-5
    assert rel_l2(V, V_or) < 1e-5
    assert rel_l2(V, V64) < 2e-6


@pytest.mark.parametrize("nz", [40, 130, 256])
def test_tensor_core_sliced_updates_match_the_double_float_factor(nz):
    """chol_df = 3: the trailing updates of the double-float Cholesky run on the tensor cores
    (eight 7-bit BF16 slices per panel value, every level of slice products summed exactly in
    FP32 tensor memory).  The factor matches the default double-float one to FP64 class and
    the inversion the oracle's 1e-5."""
    from paper_0905_0238_gb300 import Config, Solver, EDT_MIXED
    wl = small_workload(nx=32, nz=nz, nf=4, alpha=1e-2, dz=8.0)
    D = born_data(wl, salt=9)
    V_or, _ = edt2d.invert(wl, D.astype(np.complex128))
    out = {}
    for cd in (0, 3):
        s = Solver(Config.from_workload(wl, precision=EDT_MIXED, passes=3, refine=1, chol_df=cd))
        V = s.invert(dev(D)).cpu().numpy()
        st = s.stats()
        assert st.n_notpd == 0 and st.n_nonfinite == 0 and st.gram_timeouts == 0
        out[cd] = (V, np.tril(s.factor().cpu().numpy()))
    L0, L3 = out[0][1], out[3][1]
    assert np.abs(L3 - L0).max() <= 1e-12 * np.abs(L0).max()
    assert rel_l2(out[3][0], V_or) < 1e-5
