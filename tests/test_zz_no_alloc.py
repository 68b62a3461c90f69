"""The allocation-free depth march matches the oracle and the workspace-based one.

edt_green_noalloc exists for callers that may not allocate device memory; it keeps its
scratch in a fixed array inside the library.  This file is collected last so that a run
stopping at its first failure has already run every other test; it must pass on its own
in a fresh process as well as after the rest of the suite.
"""
import numpy as np
import pytest

import synth
from oracle import edt2d
from tests.gpu_helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(wl, out):
    from paper_0905_0238_gb300 import edt
    edt.edt_green_noalloc(wl.nx, wl.dx, wl.nz, wl.dz, wl.z0, wl.freq_hz, wl.eps,
                          wl.layer_top, wl.layer_vel, out.data_ptr(),
                          torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("name,nfreq", [("small_2d", 32), ("production_2d", 128)])
def test_green_noalloc_matches_green_twice(name, nfreq):
    """Two calls in a row (sharing the scratch array) against edt_green and, on sampled
    frequencies, against the oracle's table."""
    from paper_0905_0238_gb300 import Config, Solver, EDT_FP64
    wl = synth.preset(name)
    wl.freq_hz = wl.freq_hz[:nfreq]
    ref = Solver(Config.from_workload(wl, precision=EDT_FP64)).green()
    torch.cuda.synchronize()
    fs = np.unique([0, nfreq // 2, nfreq - 1])
    wl_s = synth.preset(name)
    wl_s.freq_hz = wl.freq_hz[fs]
    want = edt2d.green_table(wl_s)[:, : wl.nx // 2 + 1, :]
    out = torch.empty_like(ref)
    for _ in range(2):
        out.fill_(float("nan"))
        _noalloc(wl, out)
        torch.cuda.synchronize()
        assert torch.isfinite(out.real).all() and torch.isfinite(out.imag).all()
        got = out.cpu().numpy()
        assert rel_l2(got, ref.cpu().numpy()) < 1e-12
        assert rel_l2(got[fs], want) < 1e-12


def test_green_noalloc_one_frequency_per_chunk():
    """nx = 2048 with 73 layers: one frequency's recursion coefficients (1025 * 73 * 112
    bytes) nearly fill the 8 MiB scratch, so each of the three frequencies is its own chunk;
    the table matches the oracle on two calls in a row."""
    tops = np.arange(73) * 20.0
    vel = np.linspace(1500.0, 3600.0, 73)
    wl = synth.Workload("chunk1", nx=2048, dx=12.5, freq_hz=np.array([4.0, 17.0, 41.0]), eps=0.15,
                        nz=16, dz=50.0, z0=0.0, layer_top=tops, layer_vel=vel, alpha=1e-2,
                        cutoff=1.0)
    assert 1025 * 73 * 112 > (8 << 20) // 2
    want = edt2d.green_table(wl)[:, :1025, :]
    out = torch.empty((3, 1025, 16), dtype=torch.complex128, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        _noalloc(wl, out)
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), want) < 1e-12


def test_green_noalloc_refuses_stream_capture():
    """The call stages host arrays through pageable copies, so it refuses to be captured."""
    from paper_0905_0238_gb300 import edt
    wl = synth.preset("small_2d")
    out = torch.empty((len(wl.freq_hz), wl.nx // 2 + 1, wl.nz), dtype=torch.complex128, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        with pytest.raises(edt.EdtError) as ei:
            _noalloc(wl, out)
    assert ei.value.code == edt.EDT_EINVAL
    out.fill_(float("nan"))
    _noalloc(wl, out)                 # outside capture it runs normally afterwards
    torch.cuda.synchronize()
    assert torch.isfinite(out.real).all()
