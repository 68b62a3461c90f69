"""Host logic of the streaming solver, without a GPU: request validation, the device bytes a
request occupies, and the admission plan that cuts a request list into batches that fit one
arena of device memory."""
import copy

import numpy as np
import pytest

from synth import stream
from paper_0905_0238_gb300 import edt


def test_request_bytes_grow_with_the_request():
    base = stream.stream_requests(1, salt=20)[0]
    b0 = edt.edt_stream_request_bytes(base)
    bigger = copy.deepcopy(base)
    bigger.nz = min(512, base.nz + 128)
    assert edt.edt_stream_request_bytes(bigger) > b0
    fewer = copy.deepcopy(base)
    fewer.rows, fewer.data = base.rows[:64], base.data[:64]
    assert edt.edt_stream_request_bytes(fewer) < b0
    # the G matrix (FP64 + FP32 copy) alone is 12 nz^2 bytes
    assert b0 > 12 * base.nz ** 2


@pytest.mark.parametrize("bad", ["nz0", "nz513", "top", "vel", "row", "freq", "layers"])
def test_invalid_requests_are_rejected(bad):
    s = copy.deepcopy(stream.stream_requests(1, salt=21)[0])
    if bad == "nz0":
        s.nz = 0
    elif bad == "nz513":
        s.nz = 513
    elif bad == "top":
        s.layer_top = s.layer_top + 1.0
    elif bad == "vel":
        s.layer_vel = -s.layer_vel
    elif bad == "row":
        s.rows = s.rows.copy()
        s.rows[3, 2] = len(s.kval)
    elif bad == "freq":
        s.freq_hz = np.zeros_like(s.freq_hz)
    else:
        s.layer_top = np.arange(65, dtype=np.float64) * 10.0
        s.layer_vel = np.full(65, 2000.0)
    with pytest.raises(edt.EdtError) as e:
        edt.edt_stream_request_bytes(s)
    assert e.value.code == edt.EDT_EINVAL


def test_admission_plan_is_fifo_and_fits_the_arena():
    subs = stream.stream_requests(64, salt=22)
    rb = np.array([edt.edt_stream_request_bytes(s) for s in subs])
    arena = int(rb.max() * 3)
    for max_batch in (1, 5, 64):
        nb, of = edt.edt_stream_plan(rb, arena, max_batch)
        assert of[0] == 0 and np.all(np.diff(of) >= 0) and np.all(np.diff(of) <= 1)
        assert of[-1] == nb - 1
        for b in range(nb):
            sel = of == b
            assert sel.sum() <= max_batch
            assert rb[sel].sum() + 64 * 1024 <= arena
        # greedy: no batch could have taken the first request of the next one
        for b in range(nb - 1):
            sel = of == b
            nxt = np.argmax(of == b + 1)
            assert sel.sum() == max_batch or rb[sel].sum() + rb[nxt] + 64 * 1024 > arena


def test_admission_plan_edge_cases():
    assert edt.edt_stream_plan([], 1 << 30, 8)[0] == 0
    with pytest.raises(edt.EdtError) as e:
        edt.edt_stream_plan([10, 1 << 40, 10], 1 << 30, 8)
    assert e.value.code == edt.EDT_ENOMEM_WS
    with pytest.raises(edt.EdtError) as e:
        edt.edt_stream_plan([10], 1 << 30, 0)
    assert e.value.code == edt.EDT_EINVAL


def test_request_marshalling_round_trips():
    """The ctypes view of a request carries every field and array of the Python request."""
    subs = stream.stream_requests(3, salt=23)
    arr, keep = edt._sub1d_array(subs)
    for s, e in zip(subs, arr):
        assert (e.nz, e.nlayer, e.nfreq, e.nk, e.nrow) == (s.nz, len(s.layer_top), len(s.freq_hz), len(s.kval), s.nrow)
        assert (e.dz, e.z0, e.eps, e.alpha, e.dx) == (s.dz, s.z0, s.eps, s.alpha, s.dx)
        np.testing.assert_array_equal(np.ctypeslib.as_array(e.layer_top_m, (e.nlayer,)), s.layer_top)
        np.testing.assert_array_equal(np.ctypeslib.as_array(e.layer_vel_mps, (e.nlayer,)), s.layer_vel)
        np.testing.assert_array_equal(np.ctypeslib.as_array(e.freq_hz, (e.nfreq,)), s.freq_hz)
        np.testing.assert_array_equal(np.ctypeslib.as_array(e.kval, (e.nk,)), s.kval)
        np.testing.assert_array_equal(np.ctypeslib.as_array(e.rows, (e.nrow, 3)), s.rows)
        d = np.ctypeslib.as_array(e.data, (e.nrow, 4))
        np.testing.assert_array_equal(d[:, 0] + 1j * d[:, 1], s.data[:, 0])
        np.testing.assert_array_equal(d[:, 2] + 1j * d[:, 3], s.data[:, 1])
