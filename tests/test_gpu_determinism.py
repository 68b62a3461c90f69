"""Repeated calls give the same bits.

Every sum across CTAs on the inversion paths runs in a fixed order: the Gram's trace (per
producer warp and segment, added by the reduction in slot order), the refinement's residual
(per CTA, added in CTA order), and the streaming path's trace and residual likewise.  So the
same input gives bitwise the same output, call after call, whatever ran in between and
however the CTAs were scheduled.
"""
import numpy as np
import pytest

import synth
from synth import stream
from oracle import edt2d, stream1d
from tests.gpu_helpers import small_workload, blobs, dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _line_data(wl, salt):
    D = edt2d.forward(wl, blobs(wl, salt=salt))
    D = D + synth.noise_snr(synth.rng_for(6, salt=salt), D, 20.0)
    return np.ascontiguousarray(D.astype(np.complex64))


@pytest.mark.parametrize("alpha,refine", [(1e-2, 1), (1e-5, 2)])
def test_line_mixed_repeats_bitwise(alpha, refine):
    from paper_0905_0238_gb300 import Config, Solver, EDT_MIXED
    wl = small_workload(nx=64, nz=40, nf=6, alpha=alpha, dz=8.0)
    s = Solver(Config.from_workload(wl, precision=EDT_MIXED, refine=refine))
    D, D2 = dev(_line_data(wl, 1)), dev(_line_data(wl, 2))
    V0 = s.invert(D).cpu().numpy()
    for _ in range(3):
        s.invert(D2)                     # another problem in between
        assert np.array_equal(s.invert(D).cpu().numpy(), V0)
    assert np.array_equal(Solver(s.cfg).invert(D).cpu().numpy(), V0)   # a fresh context


def test_line_mixed_full_size_repeats_bitwise():
    """512 midpoints, 256 depths, 128 frequencies (the benchmark's line)."""
    from paper_0905_0238_gb300 import Config, Solver, EDT_MIXED
    wl = synth.preset("production_2d")
    rng = synth.rng_for(8, salt=3)
    D = dev((rng.standard_normal((len(wl.freq_hz), wl.nx, wl.nx))
             + 1j * rng.standard_normal((len(wl.freq_hz), wl.nx, wl.nx))).astype(np.complex64))
    s = Solver(Config.from_workload(wl, precision=EDT_MIXED))
    V0 = s.invert(D).cpu().numpy()
    for _ in range(2):
        assert np.array_equal(s.invert(D).cpu().numpy(), V0)


def test_window_repeats_bitwise():
    from paper_0905_0238_gb300 import Config, Solver
    tops, vel = synth.layers_gradient_staircase(1500.0, 3000.0, 160.0, 10.0, sub=2)
    wl = synth.Workload3D("t", nx=32, ny=32, dx=10.0, dy=10.0, wx=4, wy=4,
                          freq_hz=synth.freqs_uniform(4, 10.0, 40.0), eps=0.15, nz=16, dz=10.0,
                          z0=0.0, layer_top=tops, layer_vel=vel, alpha=1e-4, cutoff=1.0)
    rng = synth.rng_for(9, salt=4)
    s = Solver(Config.from_workload(wl))
    shape = s.cfg.data_shape(len(wl.freq_hz))
    D = dev((rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64))
    V0 = s.invert(D).cpu().numpy()
    for _ in range(2):
        assert np.array_equal(s.invert(D).cpu().numpy(), V0)


def test_stream_repeats_bitwise():
    from paper_0905_0238_gb300 import Stream
    rng = synth.rng_for(4, salt=990)
    subs = []
    for nz, nr, nl in ((64, 300, 5), (200, 2048, 20), (512, 4096, 9), (33, 1, 2)):
        sub = stream.sub1d_random(rng, nz_range=(nz, nz), rows_range=(nr, nr), layers_range=(nl, nl))
        if sub.nrow:
            d = stream1d.kernel_rows(sub) @ rng.standard_normal((sub.nz, 2))
            sd = np.sqrt(np.mean(np.abs(d) ** 2) / 200.0)
            sub.data = (d + sd * (rng.standard_normal(d.shape)
                                  + 1j * rng.standard_normal(d.shape))).astype(np.complex64)
        subs.append(sub)
    st = Stream(max_batch=4)
    v0, s0 = st.solve(subs)
    assert list(s0) == [0] * len(subs)
    for _ in range(2):
        st.solve(subs[::-1])             # the same requests in another batch order
        v, s = st.solve(subs)
        assert list(s) == [0] * len(subs)
        for a, b in zip(v, v0):
            assert np.array_equal(a, b)
