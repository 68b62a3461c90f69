"""The partitioned solve on the GPU: every rank of a 2- or 4-rank partition run in turn in one
process (the collectives by the in-process group), through the C ABI's export, import,
solve-imported and inverse entry points.

FP64 path: the same systems in the same arithmetic as one context, so V equals edt_invert's
to rounding and the oracle's to the FP64 tolerance.  Mixed path: each rank's tensor-core Gram
splits its rows differently, so V is compared with the oracle at the mixed tolerance.
"""
import numpy as np
import pytest

import synth
from oracle import edt2d
from tests.gpu_helpers import rel_l2, small_workload, blobs, dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _data(wl, salt, dtype=np.complex128):
    D = edt2d.forward(wl, blobs(wl, salt=salt))
    D = D + synth.noise_snr(synth.rng_for(2, salt=100 + salt), D, 25.0)
    return np.ascontiguousarray(D.astype(dtype))


@pytest.mark.parametrize("world,nf,cutoff", [(2, 6, 1.0), (4, 7, 1.0), (3, 7, 0.5)])
def test_partition_fp64_equals_one_context_and_the_oracle(world, nf, cutoff):
    from paper_0905_0238_gb300 import Config, Solver, EDT_FP64
    from paper_0905_0238_gb300 import partition as P
    wl = small_workload(nx=32, nz=24, nf=nf, alpha=1e-3, cutoff=cutoff)
    D = _data(wl, 11)
    cfg = Config.from_workload(wl, precision=EDT_FP64)
    be = P.GpuBackend(cfg)
    fb, mb = P.plan_partition(be.sub_costs(), nf, world)
    V = P.invert_partitioned_local(be, dev(D), fb, mb).cpu().numpy()
    V1 = Solver(cfg).invert(dev(D)).cpu().numpy()
    V_or, _ = edt2d.invert(wl, D)
    assert rel_l2(V, V1) < 1e-12
    assert rel_l2(V, V_or) < 1e-10


@pytest.mark.parametrize("world", [2, 4])
def test_partition_mixed_matches_the_oracle(world):
    from paper_0905_0238_gb300 import Config, EDT_MIXED
    from paper_0905_0238_gb300 import partition as P
    wl = small_workload(nx=32, nz=40, nf=8, alpha=1e-2, dz=8.0)
    D = _data(wl, 12, np.complex64)
    cfg = Config.from_workload(wl, precision=EDT_MIXED, passes=3, refine=1)
    be = P.GpuBackend(cfg)
    fb, mb = P.plan_partition(be.sub_costs(), len(wl.freq_hz), world)
    V = P.invert_partitioned_local(be, dev(D), fb, mb).cpu().numpy()
    V_or, _ = edt2d.invert(wl, D.astype(np.complex128))
    assert rel_l2(V, V_or) < 1e-5


@pytest.mark.parametrize("world", [2, 4])
def test_partition_full_size_matches_one_context(world):
    """512 midpoints, 256 depths, 128 frequencies (the 2D line the benchmark times; Born data of
    a 3 % random field plus 20 dB noise): the partitioned FP64 path equals one FP64 context to
    rounding, the partitioned mixed path one mixed context to its tolerance."""
    from paper_0905_0238_gb300 import Config, Solver, EDT_MIXED, EDT_FP64
    from paper_0905_0238_gb300 import partition as P
    wl = synth.preset("production_2d")
    V = synth.perturbation_random_field(synth.rng_for(1, salt=5), wl.nx, wl.dx, wl.nz, wl.dz,
                                        wl.z0, wl.layer_top, wl.layer_vel, corr=40.0, rms=0.03)
    fp64 = Solver(Config.from_workload(wl, precision=EDT_FP64))
    D = fp64.forward(torch.from_numpy(V).cuda(), out_dtype=torch.complex64)
    gen = torch.Generator(device=D.device)
    gen.manual_seed(synth.SEED_BASE + 905)
    sd = torch.sqrt((D.abs() ** 2).mean(dim=(1, 2), keepdim=True) / 10 ** (wl.snr_db / 10) / 2)
    D = (D + torch.complex(torch.randn(D.shape, device=D.device, generator=gen),
                           torch.randn(D.shape, device=D.device, generator=gen)) * sd).contiguous()
    for cfg, tol in ((Config.from_workload(wl, precision=EDT_FP64), 1e-12),
                     (Config.from_workload(wl, precision=EDT_MIXED, passes=3, refine=1), 1e-6)):
        be = P.GpuBackend(cfg)
        fb, mb = P.plan_partition(be.sub_costs(), len(wl.freq_hz), world)
        Vp = P.invert_partitioned_local(be, D, fb, mb).cpu().numpy()
        V1 = Solver(cfg).invert(D).cpu().numpy()
        assert rel_l2(Vp, V1) < tol, cfg.precision


def test_import_refuses_a_block_of_the_wrong_size():
    from paper_0905_0238_gb300 import Config, Solver, EDT_FP64, EdtError, EDT_EINVAL
    from paper_0905_0238_gb300 import edt
    wl = small_workload(nx=16, nz=12, nf=4, alpha=1e-3)
    s = Solver(Config.from_workload(wl, precision=EDT_FP64, sub_begin=2, sub_end=5))
    off = edt.edt_row_offsets(s.ctx, s.nsub)
    assert np.all(np.diff(off)[:2] == 0) and np.all(np.diff(off)[5:] == 0)
    n = int(off[-1])
    blk = torch.zeros((n, 2), dtype=torch.complex128, device=s.device)
    edt.edt_import_rhs(s.ctx, blk.data_ptr(), n, 0, 4, s._stream())
    with pytest.raises(EdtError) as e:
        edt.edt_import_rhs(s.ctx, blk.data_ptr(), n - 1, 0, 4, s._stream())
    assert e.value.code == EDT_EINVAL
