"""GB300-native extended diffraction tomography: batched 1D depth inversions per midpoint
wavenumber behind a C ABI (``include/edt.h``), with hand-written sm_103a CUDA kernels.

Python side: :mod:`paper_0905_0238_gb300.edt` (ctypes binding and a workspace-owning
``Solver``) and :mod:`paper_0905_0238_gb300.build` (in-tree nvcc build of ``libedt.so``).
"""
from .edt import *  # noqa: F401,F403
from .edt import Config, Solver, EdtError, Stream  # noqa: F401
