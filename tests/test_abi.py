"""The C-ABI library builds, loads and exports every entry point declared in include/edt.h."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "edt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(edt_[a-z_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_0905_0238_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    syms = declared_symbols()
    assert len(syms) >= 14
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing


def test_host_side_validation_without_gpu():
    """edt_create is host-only: invalid configurations are rejected with status codes."""
    import numpy as np
    from paper_0905_0238_gb300 import edt
    freq = np.array([5.0, 10.0]); top = np.array([0.0, 100.0]); vel = np.array([1500.0, 2000.0])
    dp = ctypes.POINTER(ctypes.c_double)

    def cfg(**kw):
        base = dict(nx=32, dx=10.0, nz=16, dz=10.0, z0=0.0, nfreq=2, freq_hz=freq.ctypes.data_as(dp),
                    eps=0.15, nlayer=2, layer_top_m=top.ctypes.data_as(dp),
                    layer_vel_mps=vel.ctypes.data_as(dp), precision=edt.EDT_FP64, passes=1,
                    refine=1, alpha=1e-3, cutoff=1.0, fold=1)
        base.update(kw)
        return edt.edt_config(**base)

    ctx, ws = edt.edt_create(cfg())
    assert ws > 0
    counts = edt.edt_row_counts(ctx, 17)
    assert counts.shape == (17,) and counts.min() >= 0
    st = edt.edt_get_stats(ctx)
    assert st.n_sub == 17 and st.rows_total == counts.sum() and st.rows_solved <= st.rows_total
    edt.edt_destroy(ctx)
    # the transform chunk: every frequency when they fit, else the requested plane count
    for req, want in ((0, None), (1, 1), (2, 2), (3, None), (10 ** 6, None)):
        ctx, ws_req = edt.edt_create(cfg(freq_chunk=req))
        st = edt.edt_get_stats(ctx)
        assert st.freq_chunk == (want if want is not None else cfg().nfreq)
        edt.edt_destroy(ctx)
    for bad, code in ((dict(nx=48), edt.EDT_EUNSUPPORTED), (dict(dx=-1.0), edt.EDT_EINVAL),
                      (dict(precision=7), edt.EDT_EINVAL), (dict(fold=3), edt.EDT_EINVAL),
                      (dict(precision=edt.EDT_MIXED, passes=2), edt.EDT_EINVAL),
                      (dict(precision=edt.EDT_MIXED, nz=300), edt.EDT_EUNSUPPORTED),
                      (dict(chol_df=4), edt.EDT_EINVAL), (dict(freq_chunk=-1), edt.EDT_EINVAL)):
        with pytest.raises(edt.EdtError) as ei:
            edt.edt_create(cfg(**bad))
        assert ei.value.code == code


@pytest.mark.parametrize("name", ["small_2d", "production_2d", "paper_2d"])
def test_host_row_plan_matches_oracle_cut(name):
    """The library's per-wavenumber row counts equal the oracle's evanescent cut."""
    import numpy as np
    import synth
    from oracle import edt2d
    from paper_0905_0238_gb300 import edt
    wl = synth.preset(name)
    freq = np.ascontiguousarray(wl.freq_hz); top = np.ascontiguousarray(wl.layer_top)
    vel = np.ascontiguousarray(wl.layer_vel)
    dp = ctypes.POINTER(ctypes.c_double)
    for fold in (0, 1):
        c = edt.edt_config(nx=wl.nx, dx=wl.dx, nz=wl.nz, dz=wl.dz, z0=wl.z0, nfreq=len(freq),
                           freq_hz=freq.ctypes.data_as(dp), eps=wl.eps, nlayer=len(top),
                           layer_top_m=top.ctypes.data_as(dp), layer_vel_mps=vel.ctypes.data_as(dp),
                           precision=edt.EDT_FP64, passes=1, refine=1, alpha=wl.alpha,
                           cutoff=wl.cutoff, fold=fold)
        ctx, _ = edt.edt_create(c)
        counts = edt.edt_row_counts(ctx, wl.nx // 2 + 1)
        st = edt.edt_get_stats(ctx)
        edt.edt_destroy(ctx)
        ms = range(0, wl.nx // 2 + 1, 1 if wl.nx <= 64 else 37)
        for m in ms:
            assert counts[m] == len(edt2d.kept_rows(wl, m)), (name, m)
        if fold == 0:
            assert st.rows_solved == st.rows_total
        else:
            # reciprocal pairs merge: at least half the rows remain, at most all of them
            assert st.rows_total / 2 <= st.rows_solved < st.rows_total


def test_tuning_is_validated_and_kept_without_gpu():
    """Launch shapes: defaults, a valid change is kept, invalid values are rejected."""
    import numpy as np
    from paper_0905_0238_gb300 import edt
    import synth
    wl = synth.preset("production_2d")
    dp = ctypes.POINTER(ctypes.c_double)
    fr = np.ascontiguousarray(wl.freq_hz); tp = np.ascontiguousarray(wl.layer_top)
    vl = np.ascontiguousarray(wl.layer_vel)
    cfg = edt.edt_config(nx=wl.nx, dx=wl.dx, nz=wl.nz, dz=wl.dz, z0=wl.z0, nfreq=len(fr),
                         freq_hz=fr.ctypes.data_as(dp), eps=wl.eps, nlayer=len(tp),
                         layer_top_m=tp.ctypes.data_as(dp), layer_vel_mps=vl.ctypes.data_as(dp),
                         precision=edt.EDT_MIXED, passes=3, refine=1, alpha=wl.alpha,
                         cutoff=wl.cutoff, fold=1)
    ctx, ws0 = edt.edt_create(cfg)
    t = edt.edt_get_tuning(ctx)
    assert (t.band_budget_mb, t.band_cols, t.refine_shape, t.window_ztile, t.overlap) == (48, 8, 0, 4, 1)
    st0 = edt.edt_get_stats(ctx)
    t.band_budget_mb, t.band_cols, t.refine_shape = 16, 4, 2
    edt.edt_set_tuning(ctx, t)
    t2 = edt.edt_get_tuning(ctx)
    assert (t2.band_budget_mb, t2.band_cols, t2.refine_shape) == (16, 4, 2)
    st = edt.edt_get_stats(ctx)
    assert st.workspace_bytes == st0.workspace_bytes       # sized for every candidate
    assert st.freq_chunk <= st0.freq_chunk                 # smaller budget, smaller chunks
    for field, bad in (("band_budget_mb", 20), ("band_cols", 6), ("refine_shape", 4), ("window_ztile", 3),
                       ("overlap", 2)):
        tb = edt.edt_get_tuning(ctx)
        setattr(tb, field, bad)
        with pytest.raises(edt.EdtError) as ei:
            edt.edt_set_tuning(ctx, tb)
        assert ei.value.code == edt.EDT_EINVAL
    edt.edt_destroy(ctx)


def test_solver_variant_validation_without_gpu():
    """Truncated SVD and the vertical-wavenumber disk: FP64 line path only, TSVD up to 96
    depths; invalid values are rejected before any device work."""
    import numpy as np
    from paper_0905_0238_gb300 import edt
    freq = np.array([5.0, 10.0]); top = np.array([0.0, 100.0]); vel = np.array([1500.0, 2000.0])
    dp = ctypes.POINTER(ctypes.c_double)

    def code(**kw):
        base = dict(nx=32, dx=10.0, nz=16, dz=10.0, z0=0.0, nfreq=2, freq_hz=freq.ctypes.data_as(dp),
                    eps=0.15, nlayer=2, layer_top_m=top.ctypes.data_as(dp),
                    layer_vel_mps=vel.ctypes.data_as(dp), precision=edt.EDT_FP64, passes=1,
                    refine=1, alpha=1e-3, cutoff=1.0, fold=1)
        base.update(kw)
        ctx, ws = ctypes.c_void_p(), ctypes.c_size_t()
        rc = edt._lib().edt_create(ctypes.byref(ctx), ctypes.byref(edt.edt_config(**base)), ctypes.byref(ws))
        if ctx.value:
            edt._lib().edt_destroy(ctx)
        return rc, ws.value

    assert code(solver=1, tsvd_tol=-1e-3)[0] == edt.EDT_OK
    assert code(solver=1, nz=97)[0] == edt.EDT_EUNSUPPORTED
    assert code(solver=1, precision=edt.EDT_MIXED, passes=3)[0] == edt.EDT_EUNSUPPORTED
    assert code(kz_disk=2.2, precision=edt.EDT_MIXED, passes=3)[0] == edt.EDT_EUNSUPPORTED
    assert code(kz_disk=-1.0)[0] == edt.EDT_EINVAL
    assert code(solver=2)[0] == edt.EDT_EINVAL
    rc0, ws0 = code()
    rc1, ws1 = code(kz_disk=2.2)
    assert rc0 == rc1 == edt.EDT_OK and ws1 > ws0


def test_disk_plan_matches_the_oracle_without_gpu():
    """The host plan of the vertical-wavenumber disk keeps, for every midpoint index, the same
    number of depth-basis columns as the oracle's disk (same basis order, same inequality)."""
    import numpy as np
    import synth
    from oracle import edt2d
    from paper_0905_0238_gb300 import edt
    dp = ctypes.POINTER(ctypes.c_double)
    for wl, factor in ((synth.preset("paper_2d"), 1.2), (synth.preset("small_2d"), 0.7)):
        fr = np.ascontiguousarray(wl.freq_hz, dtype=np.float64)
        top = np.ascontiguousarray(wl.layer_top, dtype=np.float64)
        vel = np.ascontiguousarray(wl.layer_vel, dtype=np.float64)
        cfg = edt.edt_config(nx=wl.nx, dx=wl.dx, nz=wl.nz, dz=wl.dz, z0=wl.z0, nfreq=len(fr),
                             freq_hz=fr.ctypes.data_as(dp), eps=wl.eps, nlayer=len(top),
                             layer_top_m=top.ctypes.data_as(dp), layer_vel_mps=vel.ctypes.data_as(dp),
                             precision=edt.EDT_FP64, passes=1, refine=0, alpha=wl.alpha,
                             cutoff=wl.cutoff, fold=1, kz_disk=factor)
        ctx, ws = ctypes.c_void_p(), ctypes.c_size_t()
        assert edt._lib().edt_create(ctypes.byref(ctx), ctypes.byref(cfg), ctypes.byref(ws)) == edt.EDT_OK
        try:
            got = edt.edt_kz_disk_columns(ctx, wl.nx // 2 + 1)
        finally:
            edt._lib().edt_destroy(ctx)
        want = [int(edt2d.kz_disk_keep(wl, m, factor).sum()) for m in range(wl.nx // 2 + 1)]
        assert list(got) == want
        assert min(want) < wl.nz          # the disk removes columns on these shapes


def test_green_noalloc_rejects_oversized_coefficients_without_gpu():
    """One frequency's recursion coefficients ((nx/2+1) * nlayer * 112 bytes) must fit the
    allocation-free call's 8 MiB scratch: nx = 2048 with 74 layers needs 8.5 MB and is refused
    on the host, before any device call (nothing is launched)."""
    import numpy as np
    from paper_0905_0238_gb300 import edt
    tops = np.arange(74) * 20.0
    vel = np.linspace(1500.0, 3600.0, 74)
    assert 1025 * 74 * 112 > (8 << 20)
    with pytest.raises(edt.EdtError) as ei:
        edt.edt_green_noalloc(2048, 12.5, 16, 50.0, 0.0, np.array([10.0]), 0.15, tops, vel,
                              0x1000, 0)
    assert ei.value.code == edt.EDT_EUNSUPPORTED
    with pytest.raises(edt.EdtError) as ei:
        edt.edt_green_noalloc(48, 12.5, 16, 50.0, 0.0, np.array([10.0]), 0.15, tops, vel, 0x1000, 0)
    assert ei.value.code == edt.EDT_EINVAL


def test_wait_test_hook_validates_on_the_host():
    """edt_set_wait_test is host-only: a stall needs a positive budget; negative budgets and
    other stall values are refused."""
    import numpy as np
    from paper_0905_0238_gb300 import edt
    freq = np.array([5.0, 10.0]); top = np.array([0.0, 100.0]); vel = np.array([1500.0, 2000.0])
    dp = ctypes.POINTER(ctypes.c_double)
    cfg = edt.edt_config(nx=32, dx=10.0, nz=16, dz=10.0, z0=0.0, nfreq=2, freq_hz=freq.ctypes.data_as(dp),
                         eps=0.15, nlayer=2, layer_top_m=top.ctypes.data_as(dp),
                         layer_vel_mps=vel.ctypes.data_as(dp), precision=edt.EDT_MIXED, passes=3,
                         refine=1, alpha=1e-2, cutoff=1.0, fold=1)
    ctx, _ = edt.edt_create(cfg)
    try:
        edt.edt_set_wait_test(ctx, 1000, True)
        edt.edt_set_wait_test(ctx, 0, False)
        for cyc, stall in ((0, True), (-1, False)):
            with pytest.raises(edt.EdtError) as ei:
                edt.edt_set_wait_test(ctx, cyc, stall)
            assert ei.value.code == edt.EDT_EINVAL
    finally:
        edt.edt_destroy(ctx)


def test_ranged_and_sharded_row_plans_without_gpu():
    """A context over a subproblem range plans the full plan's rows inside it and none outside;
    contexts over contiguous frequency shards plan, per subproblem, row counts that add up to
    the full plan's (the oracle's cut restricted to each shard); the import refuses a block
    whose row count differs from the context's before touching any device memory."""
    import numpy as np
    import synth
    from oracle import edt2d
    from paper_0905_0238_gb300 import edt, Config
    from paper_0905_0238_gb300.partition import GpuBackend, plan_partition
    wl = synth.preset("small_2d")
    nsub = wl.nx // 2 + 1
    full = GpuBackend(Config.from_workload(wl, precision=edt.EDT_FP64, fold=0)).sub_rows()
    assert [int(x) for x in full] == [len(edt2d.kept_rows(wl, m)) for m in range(nsub)]
    for prec in (edt.EDT_FP64, edt.EDT_MIXED):
        base = Config.from_workload(wl, precision=prec)
        rows = GpuBackend(base).sub_rows()
        fb, mb = plan_partition(rows, len(wl.freq_hz), 3)
        for r in range(3):
            c, _arrays = Config.from_workload(wl, precision=prec, sub_begin=mb[r],
                                              sub_end=mb[r + 1]).c_config()
            ctx, _ = edt.edt_create(c)
            try:
                got = np.diff(edt.edt_row_offsets(ctx, nsub))
                with pytest.raises(edt.EdtError) as ei:       # no workspace: refused first
                    edt.edt_import_rhs(ctx, 0, 0, 0, 1, 0)
                assert ei.value.code == edt.EDT_ENOMEM_WS
            finally:
                edt.edt_destroy(ctx)
            want = np.where((np.arange(nsub) >= mb[r]) & (np.arange(nsub) < mb[r + 1]), rows, 0)
            assert np.array_equal(got, want)
        shard_sum = np.zeros(nsub, dtype=np.int64)
        for r in range(3):
            c, _arrays = Config.from_workload(
                wl, precision=prec, freq_hz=list(wl.freq_hz)[fb[r]:fb[r + 1]]).c_config()
            ctx, _ = edt.edt_create(c)
            try:
                shard_sum += np.diff(edt.edt_row_offsets(ctx, nsub))
            finally:
                edt.edt_destroy(ctx)
        assert np.array_equal(shard_sum, rows)
    for b, e in ((3, 2), (0, nsub + 1), (-1, 2)):
        c, _arrays = Config.from_workload(wl, sub_begin=b, sub_end=e).c_config()
        with pytest.raises(edt.EdtError) as ei:
            edt.edt_create(c)
        assert ei.value.code == edt.EDT_EINVAL
