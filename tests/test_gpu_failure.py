"""Failure detection of the bounded device waits, exercised without a GPU fault.

Every wait of the two tensor-core Gram kernels is bounded.  The test hook
(edt_set_wait_test / edt_stream_set_wait_test) shortens the budget to about a millisecond and
makes the MMA issuer wait on an mbarrier that nothing completes, so the wait runs out the way a
lost producer signal would: the kernel raises its device flag, releases its producers through
its abort flag, drains what it issued, frees its tensor memory and returns.  The host then reads
EDT_ETIMEOUT (edt_get_stats on the line path, the per-request status on the streaming path),
and the same context solves the next call correctly.  Nothing traps and nothing waits forever.
"""
import numpy as np
import pytest

import synth
from oracle import edt2d, stream1d
from synth import stream
from tests.gpu_helpers import rel_l2, small_workload, blobs, dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BUDGET = 2_000_000          # clock cycles: about 1 ms at the GB300's SM clock


def test_line_gram_timeout_surfaces_and_the_context_recovers():
    from paper_0905_0238_gb300 import Config, Solver, EDT_MIXED, EDT_ETIMEOUT, EDT_OK
    wl = small_workload(nx=32, nz=40, nf=6, alpha=1e-2, dz=8.0)
    V = blobs(wl, salt=5)
    D = edt2d.forward(wl, V)
    D = D + synth.noise_snr(synth.rng_for(0, salt=105), D, 20.0)
    D = np.ascontiguousarray(D.astype(np.complex64))
    V_or, _ = edt2d.invert(wl, D.astype(np.complex128))
    s = Solver(Config.from_workload(wl, precision=EDT_MIXED, passes=3, refine=1))
    for _ in range(2):              # twice: the flag is cleared per call and raised again
        s.set_wait_test(BUDGET, True)
        s.invert(dev(D))
        st = s.stats()
        assert st.gram_timeouts == 1 and st.last_status == EDT_ETIMEOUT
        s.set_wait_test(0, False)
        Vg = s.invert(dev(D)).cpu().numpy()
        st = s.stats()
        assert st.gram_timeouts == 0 and st.last_status == EDT_OK
        assert rel_l2(Vg, V_or) < 1e-5


def test_stream_gram_timeout_surfaces_per_request_and_later_batches_run():
    from paper_0905_0238_gb300 import Stream, EDT_ETIMEOUT
    rng = synth.rng_for(4, salt=950)
    subs = [stream.sub1d_random(rng, nz_range=(nz, nz), rows_range=(nr, nr), layers_range=(nl, nl))
            for nz, nr, nl in ((96, 300, 6), (300, 1200, 14))]
    for sub in subs:
        a = stream1d.kernel_rows(sub)
        d = a @ rng.standard_normal((sub.nz, 2))
        sd = np.sqrt(np.mean(np.abs(d) ** 2) / 200.0)
        sub.data = (d + sd * (rng.standard_normal(d.shape) + 1j * rng.standard_normal(d.shape))).astype(np.complex64)
    st = Stream(max_batch=8)
    st.set_wait_test(BUDGET, True)
    _, status = st.solve(subs)
    assert list(status) == [EDT_ETIMEOUT] * len(subs)
    st.set_wait_test(0, False)
    v, status = st.solve(subs)
    assert list(status) == [0] * len(subs)
    for sub, got in zip(subs, v):
        assert rel_l2(got, stream1d.solve(sub)) < 1e-5
