"""Seeded synthetic inputs shared by the tests, the oracle checks and the benchmark.

This module holds geometry, reference-model, perturbation and noise generators only.
It contains none of the inversion method's arithmetic (no Green's functions, no Born
modelling, no transforms of the data, no solves), so that the oracle and the CUDA path
can both consume its output without sharing any of the method.

Workload presets follow the synthetic examples of the paper (Section "Numerical
Examples": complex frequency omega + i*eps with eps = 0.15 1/s, sources and receivers on
the surface z = 0, depth-dependent layered references) at the sizes used by this project:

  * ``small_2d``      64 x 64 sources/receivers, dx 10 m, 32 frequencies 5-40 Hz,
                      64 depths of 10 m, linear 1500-3000 m/s gradient as a staircase,
                      three Gaussian blobs (sigma 30 m, +-5 % velocity).
  * ``production_2d`` 512 x 512, dx 12.5 m, 128 frequencies 3-60 Hz, 256 depths of 8 m,
                      20 random layers, Gaussian-correlated 3 % rms random field,
                      complex Gaussian noise at 20 dB SNR per frequency.
  * ``paper_2d``      the paper's own acquisition (m, h every 50 m, 1-10 Hz) reduced to a
                      periodic line of 256 points, used as an extra paper-shaped size.

Finite-aperture presets (``preset3d``): ``small_3d`` (16 x 16 midpoints, 4 x 4 half-offsets),
``line_fa`` (a 64-point line with 16 half-offsets) and ``batched_3d`` (128 x 128 midpoints,
16 x 16 half-offsets, 64 frequencies 4-50 Hz, 200 depths of 10 m, 20 random layers).
"""
from .generators import *  # noqa: F401,F403
from .generators import __all__  # noqa: F401
