"""Streaming 1D solves on the GPU against the oracle: requests of every depth count band
(one to four 128-depth tiles, ragged), row counts from 1 to 4096, 1 to 30 layers; batches cut
by device memory; tickets waited out of order; empty and degenerate requests; a line
wavenumber restated as a request against the line path."""
import copy

import numpy as np
import pytest

import synth
from synth import stream
from oracle import edt2d, stream1d
from tests.gpu_helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def shaped(nz, nrow, nl, salt, modelled=True, **kw):
    """A request of the given shape; with ``modelled`` its data are the oracle's rows applied to a
    seeded model plus complex Gaussian noise at 20 dB (data a survey would record), otherwise the
    generator's pure-noise data."""
    rng = synth.rng_for(4, salt=300 + salt)
    sub = stream.sub1d_random(rng, nz_range=(nz, nz), rows_range=(nrow, nrow), layers_range=(nl, nl), **kw)
    if modelled and sub.nrow:
        a = stream1d.kernel_rows(sub)
        d = a @ rng.standard_normal((sub.nz, 2))
        sd = np.sqrt(np.mean(np.abs(d) ** 2) / 10 ** 2 / 2)
        sub.data = (d + sd * (rng.standard_normal(d.shape) + 1j * rng.standard_normal(d.shape))).astype(np.complex64)
    return sub


def solver(**kw):
    from paper_0905_0238_gb300 import Stream
    return Stream(**kw)


SHAPES = [(64, 128, 5), (100, 700, 12), (128, 1000, 30), (129, 333, 7), (200, 2048, 20),
          (256, 4096, 17), (300, 1500, 9), (384, 3000, 25), (512, 4096, 30), (511, 900, 6)]


def test_stream_batch_matches_oracle():
    subs = [shaped(*s, salt=i) for i, s in enumerate(SHAPES)]
    s = solver(max_batch=64)
    v, st = s.solve(subs)
    assert list(st) == [0] * len(subs)
    for sub, got in zip(subs, v):
        want = stream1d.solve(sub)
        assert rel_l2(got, want) < TOL, (sub.nz, sub.nrow, rel_l2(got, want))


def test_pure_noise_data_match_oracle_within_their_sensitivity():
    """Data that no model explains leave a residual as large as the data, and the solution's
    sensitivity to the FP32 rows grows with cond(G + lam I)^2 times that residual: the bar for
    such data is 1e-4 (modelled data above meet 1e-5)."""
    subs = [shaped(*s, salt=10 + i, modelled=False) for i, s in enumerate(SHAPES[:5])]
    v, st = solver(max_batch=64).solve(subs)
    assert list(st) == [0] * len(subs)
    for sub, got in zip(subs, v):
        assert rel_l2(got, stream1d.solve(sub)) < 1e-4


def test_batches_cut_by_memory_and_tickets_out_of_order():
    subs = [shaped(*s, salt=20 + i) for i, s in enumerate(SHAPES[:6])]
    ref, st0 = solver(max_batch=64).solve(subs)
    s = solver(max_batch=2)                       # three batches per submit, both arenas reused
    t1 = s.submit(subs[:4])
    t2 = s.submit(subs[4:])
    v2, st2, _ = s.wait(t2)
    v1, st1, _ = s.wait(t1)
    assert list(st1) + list(st2) == [0] * 6
    for a, b in zip(v1 + v2, ref):
        assert rel_l2(a, b) < 1e-12
    assert s.stats()["batches"] == 3


def test_degenerate_requests():
    base = shaped(96, 300, 4, salt=40)
    empty = copy.deepcopy(base)
    empty.rows, empty.data = base.rows[:0], base.data[:0]
    one_row = copy.deepcopy(base)
    one_row.rows, one_row.data = base.rows[:1], base.data[:1]
    one_depth = shaped(1, 200, 3, salt=41)
    one_layer = shaped(150, 400, 1, salt=42)
    subs = [empty, one_row, one_depth, one_layer, base]
    v, st = solver(max_batch=8).solve(subs)
    assert list(st) == [0] * len(subs)
    assert np.all(v[0] == 0)
    for sub, got in zip(subs[1:], v[1:]):
        assert rel_l2(got, stream1d.solve(sub)) < TOL


def test_weak_damping_matches_oracle():
    subs = [shaped(160, 2500, 10, salt=50, alpha=1e-3), shaped(320, 3500, 22, salt=51, alpha=1e-3)]
    v, st = solver(max_batch=4).solve(subs)
    assert list(st) == [0, 0]
    for sub, got in zip(subs, v):
        assert rel_l2(got, stream1d.solve(sub)) < TOL


def test_request_larger_than_an_arena_is_refused():
    from paper_0905_0238_gb300 import EdtError
    from paper_0905_0238_gb300.edt import EDT_ENOMEM_WS, edt_stream_request_bytes
    s = solver(max_batch=4)
    arena = s.stats()["arena_bytes"]
    big = shaped(512, 4096, 30, salt=60)
    big.kval = np.linspace(0.0, 0.2, 40000)      # a Green's table larger than one arena
    big.rows = big.rows.copy()
    assert edt_stream_request_bytes(big) > arena
    with pytest.raises(EdtError) as e:
        s.submit([shaped(64, 128, 5, salt=61), big])
    assert e.value.code == EDT_ENOMEM_WS
    assert s.stats()["batches"] == 0


def test_line_wavenumber_restated_matches_line_path():
    from paper_0905_0238_gb300 import Config, Solver, EDT_MIXED
    wl = synth.Workload("line", nx=64, dx=12.5, freq_hz=synth.freqs_uniform(6, 8.0, 40.0), eps=0.15,
                        nz=40, dz=8.0, z0=0.0, layer_top=np.array([0.0, 90.0, 200.0]),
                        layer_vel=np.array([1600.0, 2100.0, 2700.0]), alpha=1e-2, cutoff=1.0)
    D = synth.random_data(synth.rng_for(4, salt=70), (len(wl.freq_hz), wl.nx, wl.nx))
    line = Solver(Config.from_workload(wl, precision=EDT_MIXED))
    line.invert(torch.from_numpy(D.astype(np.complex64)).cuda())
    vh_line = line.vhat().cpu().numpy()
    D2 = edt2d.data_transform(D.astype(np.complex64).astype(np.complex128))
    subs = []
    ms = (1, 5, 17, 31)
    for m in ms:
        rows = edt2d.kept_rows(wl, m)
        dp, dm = edt2d.split_rhs(D2, m, rows)
        subs.append(stream.sub_from_line(wl, m, rows, dp, dm))
    v, st = solver(max_batch=8).solve(subs)
    assert list(st) == [0] * len(ms)
    for m, got in zip(ms, v):
        assert rel_l2(got, vh_line[m]) < 2 * TOL
