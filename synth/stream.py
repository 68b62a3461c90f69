"""Seeded generator of a stream of independent 1D depth subproblems (the streaming workload).

A request is the split system of one midpoint wavenumber k_m of its own line survey (eqs. DMV,
M and Split of Section "Two dimensions"), carried with everything that defines it: its layered
reference c0(z), its depth grid, its frequencies, the lateral wavenumbers its rows use, the rows
themselves as index triples (f, p, q) meaning the kernel row of frequency f over the
wavenumbers |k_p| and |k_q| = |k_p - k_m|, and the two right-hand sides (d_+, d_-) of every row.

Shapes follow the streaming configuration: 4096 requests arriving in Poisson bursts of 32-512,
depth counts uniform in 64-512, rows uniform in 128-4096, a random layered reference of 5-30
layers (the 20-layer generator's law over the request's own depth range), complex64 data.  The
rows of a request are bands of consecutive receiver wavenumbers, one band per frequency, as the
evanescent cut leaves them in a line survey.  The data are seeded complex Gaussian values: the
cost of a solve does not depend on them.

Only index and random-number work is done here: no Green's function, no kernel row, no solve.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List

import numpy as np

from .generators import layers_random, rng_for

__all__ = ["Sub1D", "sub1d_random", "stream_requests", "burst_schedule", "sub_from_line"]


@dataclass
class Sub1D:
    """One 1D subproblem: min ||Ahat x_+- - dhat_+-||^2 + lam ||x_+-||^2 over real x_+- (nz).

    Row r of the complex system is a_r(z) = s_f g(|k_p|, z) g(|k_q|, z) with
    (f, p, q) = rows[r], s_f = omega~_f^2 dz / dx and g the layered reference Green's function;
    Ahat stacks the real and imaginary parts of the rows, lam = alpha trace(Ahat^T Ahat).
    """
    nz: int
    dz: float
    z0: float
    eps: float
    alpha: float
    dx: float
    layer_top: np.ndarray     # [nlayer] float64, layer_top[0] = 0
    layer_vel: np.ndarray     # [nlayer] float64
    freq_hz: np.ndarray       # [nf] float64
    kval: np.ndarray          # [nk] float64, lateral wavenumbers |k| in rad/m
    rows: np.ndarray          # [R, 3] int32: (f, p, q) indices into freq_hz and kval
    data: np.ndarray          # [R, 2] complex64: (d_+, d_-)

    @property
    def nrow(self) -> int:
        return int(self.rows.shape[0])


def sub1d_random(rng: np.random.Generator, nz_range=(64, 512), rows_range=(128, 4096),
                 layers_range=(5, 30), N: int = 512, dx: float = 12.5, dz: float = 8.0,
                 fmin: float = 3.0, fmax: float = 60.0, alpha: float = 1e-2,
                 eps: float = 0.15) -> Sub1D:
    """One request with uniform depth count, row count and layer count in the given ranges."""
    nz = int(rng.integers(nz_range[0], nz_range[1] + 1))
    R = int(rng.integers(rows_range[0], rows_range[1] + 1))
    nl = int(rng.integers(layers_range[0], layers_range[1] + 1))
    tops, vel = layers_random(rng, nl, depth=nz * dz)
    m = int(rng.integers(1, N // 2))
    wmax = N // 2
    nf = max(1, -(-R // wmax))
    freqs = np.sort(rng.uniform(fmin, fmax, nf))
    widths = np.full(nf, R // nf, dtype=np.int64)
    widths[: R - int(widths.sum())] += 1
    n_p, fidx = [], []
    for f in range(nf):
        w = int(widths[f])
        lo = m // 2 - w // 2 + int(rng.integers(-4, 5))
        n_p.append(np.arange(lo, lo + w, dtype=np.int64))
        fidx.append(np.full(w, f, dtype=np.int64))
    n_p = np.concatenate(n_p)
    fidx = np.concatenate(fidx)
    n_q = n_p - m
    uniq = np.unique(np.concatenate([np.abs(n_p), np.abs(n_q)]))
    pos = {int(v): i for i, v in enumerate(uniq)}
    rows = np.stack([fidx, [pos[int(abs(v))] for v in n_p], [pos[int(abs(v))] for v in n_q]],
                    axis=1).astype(np.int32)
    kval = 2.0 * np.pi * uniq.astype(np.float64) / (N * dx)
    data = ((rng.standard_normal((R, 2)) + 1j * rng.standard_normal((R, 2))) / np.sqrt(2.0)).astype(np.complex64)
    return Sub1D(nz=nz, dz=dz, z0=0.0, eps=eps, alpha=alpha, dx=dx, layer_top=tops,
                 layer_vel=vel, freq_hz=freqs, kval=kval, rows=rows, data=data)


def stream_requests(n: int = 4096, salt: int = 0, **kw) -> List[Sub1D]:
    """The seeded stream of the streaming configuration (workload index 4)."""
    rng = rng_for(4, salt)
    return [sub1d_random(rng, **kw) for _ in range(n)]


def burst_schedule(n_total: int, rate_hz: float, burst=(32, 512), salt: int = 0):
    """Poisson arrivals of bursts: (sizes, arrival times in s from the first burst).

    Burst sizes are uniform in ``burst`` (the last one truncated so they sum to n_total);
    the gaps between bursts are exponential with mean 1 / rate_hz.
    """
    rng = rng_for(4, 100 + salt)
    sizes = []
    while sum(sizes) < n_total:
        s = int(rng.integers(burst[0], burst[1] + 1))
        sizes.append(min(s, n_total - sum(sizes)))
    gaps = rng.exponential(1.0 / rate_hz, len(sizes))
    gaps[0] = 0.0
    return np.array(sizes, dtype=np.int64), np.cumsum(gaps)


def sub_from_line(wl, m: int, rows_fp: np.ndarray, d_plus: np.ndarray, d_minus: np.ndarray) -> Sub1D:
    """The request that restates midpoint wavenumber m of a line workload ``wl``.

    ``rows_fp`` are the system's rows as (f, p) pairs on the line's N-point grid and
    ``d_plus``, ``d_minus`` their right-hand sides; the wavenumbers become the distinct
    |n'| of p and p - m (n' the signed index), so the request and the line system coincide.
    """
    N = wl.nx
    n = np.arange(N)
    signed = np.where(n <= N // 2, n, n - N)
    f = rows_fp[:, 0].astype(np.int64)
    p = rows_fp[:, 1].astype(np.int64)
    q = (p - m) % N
    ap, aq = np.abs(signed[p]), np.abs(signed[q])
    uniq = np.unique(np.concatenate([ap, aq]))
    pos = {int(v): i for i, v in enumerate(uniq)}
    rows = np.stack([f, [pos[int(v)] for v in ap], [pos[int(v)] for v in aq]], axis=1).astype(np.int32)
    kval = 2.0 * np.pi * uniq.astype(np.float64) / (N * wl.dx)
    data = np.stack([d_plus, d_minus], axis=1).astype(np.complex128)
    return Sub1D(nz=wl.nz, dz=wl.dz, z0=wl.z0, eps=wl.eps, alpha=wl.alpha, dx=wl.dx,
                 layer_top=np.asarray(wl.layer_top, dtype=np.float64),
                 layer_vel=np.asarray(wl.layer_vel, dtype=np.float64),
                 freq_hz=np.asarray(wl.freq_hz, dtype=np.float64), kval=kval, rows=rows, data=data)
