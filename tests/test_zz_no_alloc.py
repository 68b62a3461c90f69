"""The allocation-free depth march matches the workspace-based one.

edt_green_noalloc exists for callers that may not allocate device memory; it keeps its
scratch in a fixed array inside the library.  This file is collected last so that a run
stopping at its first failure has already run every other test; it must pass on its own
in a fresh process as well as after the rest of the suite.
"""
import numpy as np
import pytest

import synth
from tests.gpu_helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,nfreq", [("small_2d", 32), ("production_2d", 128)])
def test_green_noalloc_matches_green_twice(name, nfreq):
    from paper_0905_0238_gb300 import Config, Solver, EDT_FP64, edt
    wl = synth.preset(name)
    wl.freq_hz = wl.freq_hz[:nfreq]
    ref = Solver(Config.from_workload(wl, precision=EDT_FP64)).green()
    torch.cuda.synchronize()
    out = torch.empty_like(ref)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):                 # two calls in a row share the same scratch array
        out.fill_(float("nan"))
        edt.edt_green_noalloc(wl.nx, wl.dx, wl.nz, wl.dz, wl.z0, wl.freq_hz, wl.eps,
                              wl.layer_top, wl.layer_vel, out.data_ptr(), stream)
        torch.cuda.synchronize()
        assert torch.isfinite(out.real).all() and torch.isfinite(out.imag).all()
        assert rel_l2(out.cpu().numpy(), ref.cpu().numpy()) < 1e-12
