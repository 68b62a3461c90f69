"""Seeded generators for geometry, layered references, perturbations and noise.

Everything here is plain input preparation.  The quantities produced are the ones the
paper's problem statement takes as given (Section "Two dimensions": the reference c0(z),
the surface geometry, the frequencies, and the scattering potential V = 1/c^2 - 1/c0^2
that defines the synthetic truth), plus noise models for the data.
"""
from __future__ import annotations

from dataclasses import dataclass, field, asdict
from typing import List, Optional

import numpy as np

__all__ = [
    "SEED_BASE", "Workload", "preset", "freqs_uniform", "layers_gradient_staircase",
    "layers_random", "layers_two", "velocity_at", "perturbation_blobs",
    "perturbation_random_field", "perturbation_square", "noise_snr", "noise_paper",
    "random_data", "rng_for", "Workload3D", "preset3d", "perturbation_blobs_3d",
    "perturbation_random_field_3d",
]

SEED_BASE = 20260905


def rng_for(index: int, salt: int = 0) -> np.random.Generator:
    """The seeded generator of workload ``index`` (seed = 20260905 + index, plus a salt)."""
    return np.random.default_rng(SEED_BASE + int(index) + 1000 * int(salt))


@dataclass
class Workload:
    """A complete synthetic 2D problem description (SI units throughout)."""
    name: str
    nx: int
    dx: float
    freq_hz: np.ndarray
    eps: float
    nz: int
    dz: float
    z0: float
    layer_top: np.ndarray
    layer_vel: np.ndarray
    alpha: float
    cutoff: float
    snr_db: Optional[float] = None
    extra: dict = field(default_factory=dict)

    def summary(self) -> dict:
        d = {k: v for k, v in asdict(self).items() if not isinstance(v, np.ndarray)}
        d["nfreq"] = int(len(self.freq_hz))
        d["nlayer"] = int(len(self.layer_top))
        d["fmin"], d["fmax"] = float(self.freq_hz.min()), float(self.freq_hz.max())
        return d


def freqs_uniform(n: int, fmin: float, fmax: float) -> np.ndarray:
    """n frequencies uniformly spaced over [fmin, fmax] in Hz."""
    if n == 1:
        return np.array([float(fmin)])
    return np.linspace(float(fmin), float(fmax), int(n))


def layers_gradient_staircase(v_top: float, v_bot: float, depth: float, dz: float,
                              sub: int = 4):
    """A linear velocity gradient over [0, depth] as a staircase of constant layers.

    ``sub`` sublayers per depth step ``dz``; each sublayer takes the gradient's velocity at
    its midpoint.  Below ``depth`` a half-space of velocity ``v_bot``.
    """
    h = dz / sub
    n = int(round(depth / h))
    tops = np.arange(n + 1, dtype=np.float64) * h
    mids = (np.arange(n, dtype=np.float64) + 0.5) * h
    vel = v_top + (v_bot - v_top) * mids / depth
    return tops, np.concatenate([vel, [float(v_bot)]])


def layers_random(rng: np.random.Generator, nlayer: int = 20, depth: float = 2048.0,
                  vmin: float = 1500.0, vmax: float = 4500.0, jitter: float = 0.05):
    """nlayer equal-thickness layers over [0, depth]; the last one extends to infinity.

    Velocities are drawn uniform in [vmin, vmax], sorted increasing, then multiplied by
    (1 + U(-jitter, jitter)).
    """
    tops = np.arange(nlayer, dtype=np.float64) * (depth / nlayer)
    vel = np.sort(rng.uniform(vmin, vmax, nlayer))
    vel = vel * (1.0 + rng.uniform(-jitter, jitter, nlayer))
    return tops, vel


def layers_two(v1: float, v2: float, z_interface: float):
    """Two half-spaces: v1 above z_interface, v2 below (the paper's two-layer model)."""
    return np.array([0.0, float(z_interface)]), np.array([float(v1), float(v2)])


def velocity_at(z, layer_top, layer_vel):
    """Reference velocity at depth(s) z (an interface depth belongs to the layer below)."""
    idx = np.searchsorted(np.asarray(layer_top), np.asarray(z, dtype=np.float64), side="right") - 1
    idx = np.clip(idx, 0, len(layer_vel) - 1)
    return np.asarray(layer_vel)[idx]


def _depths(nz, dz, z0):
    return z0 + (np.arange(nz, dtype=np.float64) + 0.5) * dz


def _v_from_rel(rel, c0):
    """Scattering potential V = 1/c^2 - 1/c0^2 for c = c0 (1 + rel)."""
    c = c0 * (1.0 + rel)
    return 1.0 / c ** 2 - 1.0 / c0 ** 2


def perturbation_blobs(rng, nx, dx, nz, dz, z0, layer_top, layer_vel, nblob=3,
                       sigma=30.0, amp=0.05):
    """V(x, z) [nx][nz] for Gaussian blobs of relative velocity change +-amp."""
    x = np.arange(nx) * dx
    z = _depths(nz, dz, z0)
    c0 = velocity_at(z, layer_top, layer_vel)
    rel = np.zeros((nx, nz))
    for b in range(nblob):
        xc = rng.uniform(0.15, 0.85) * nx * dx
        zc = z0 + rng.uniform(0.2, 0.8) * nz * dz
        sgn = 1.0 if b % 2 == 0 else -1.0
        rel += sgn * amp * np.exp(-((x[:, None] - xc) ** 2 + (z[None, :] - zc) ** 2)
                                  / (2.0 * sigma ** 2))
    return _v_from_rel(rel, c0[None, :])


def perturbation_random_field(rng, nx, dx, nz, dz, z0, layer_top, layer_vel,
                              corr=40.0, rms=0.03):
    """V(x, z) for a Gaussian-correlated random relative velocity field of given rms."""
    white = rng.standard_normal((nx, nz))
    kx = 2 * np.pi * np.fft.fftfreq(nx, dx)
    kz = 2 * np.pi * np.fft.fftfreq(nz, dz)
    filt = np.exp(-0.25 * corr ** 2 * (kx[:, None] ** 2 + kz[None, :] ** 2))
    rel = np.real(np.fft.ifft2(np.fft.fft2(white) * filt))
    rel *= rms / max(np.sqrt(np.mean(rel ** 2)), 1e-300)
    z = _depths(nz, dz, z0)
    c0 = velocity_at(z, layer_top, layer_vel)
    return _v_from_rel(rel, c0[None, :])


def perturbation_square(nx, dx, nz, dz, z0, xc, zc, side, value=1.0):
    """The paper's square anomaly: V = value inside a square of given side, else 0."""
    x = np.arange(nx) * dx
    z = _depths(nz, dz, z0)
    inside = (np.abs(x[:, None] - xc) <= side / 2) & (np.abs(z[None, :] - zc) <= side / 2)
    return np.where(inside, float(value), 0.0)


def noise_snr(rng, D, snr_db):
    """Circular complex Gaussian noise with power = (signal power per frequency) / 10^(snr/10).

    ``D`` is [nfreq][...]; the returned array has D's shape and dtype.
    """
    D = np.asarray(D)
    axes = tuple(range(1, D.ndim))
    p_sig = np.mean(np.abs(D) ** 2, axis=axes, keepdims=True)
    p_noise = p_sig / 10.0 ** (snr_db / 10.0)
    n = (rng.standard_normal(D.shape) + 1j * rng.standard_normal(D.shape)) * np.sqrt(p_noise / 2)
    return n.astype(D.dtype)


def noise_paper(rng, D, frac=0.05):
    """The paper's noise model: per frequency, add values of modulus frac * max|D(omega)|
    with a phase uniform in [0, 2 pi)."""
    D = np.asarray(D)
    axes = tuple(range(1, D.ndim))
    amp = frac * np.max(np.abs(D), axis=axes, keepdims=True)
    ph = rng.uniform(0.0, 2 * np.pi, D.shape)
    return (amp * np.exp(1j * ph)).astype(D.dtype)


def random_data(rng, shape, dtype=np.complex128):
    """Unstructured complex Gaussian data of the given shape."""
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(dtype)


def preset(name: str) -> Workload:
    """The named workload with its seeded reference model (perturbation drawn separately)."""
    if name == "small_2d":
        tops, vel = layers_gradient_staircase(1500.0, 3000.0, 640.0, 10.0, sub=4)
        return Workload(name, nx=64, dx=10.0, freq_hz=freqs_uniform(32, 5.0, 40.0), eps=0.15,
                        nz=64, dz=10.0, z0=0.0, layer_top=tops, layer_vel=vel,
                        alpha=1e-5, cutoff=1.0, snr_db=None)
    if name == "production_2d":
        tops, vel = layers_random(rng_for(1), 20, 2048.0)
        return Workload(name, nx=512, dx=12.5, freq_hz=freqs_uniform(128, 3.0, 60.0), eps=0.15,
                        nz=256, dz=8.0, z0=0.0, layer_top=tops, layer_vel=vel,
                        alpha=1e-2, cutoff=1.0, snr_db=20.0)
    if name == "paper_2d":
        tops, vel = layers_two(1500.0, 4000.0, 1000.0)
        return Workload(name, nx=256, dx=50.0, freq_hz=freqs_uniform(10, 1.0, 10.0), eps=0.15,
                        nz=65, dz=50.0, z0=775.0, layer_top=tops, layer_vel=vel,
                        alpha=1e-3, cutoff=1.0, snr_db=None)
    raise KeyError(name)


@dataclass
class Workload3D:
    """A synthetic finite-aperture problem on an nx x ny periodic midpoint grid.

    Data D[f][my][mx][wy][wx] are recorded at midpoint (mx, my) (grid units) for every
    half-offset (wx, wy) of a wx_n x wy_n window of signed indices [-n/2, n/2): the source sits
    at midpoint - half-offset and the receiver at midpoint + half-offset, so the offsets
    are 2 (wx, wy) grid steps.  ny = 1 and wy_n = 1 give the 2D line survey with a finite
    aperture.
    """
    name: str
    nx: int
    ny: int
    dx: float
    dy: float
    wx: int
    wy: int
    freq_hz: np.ndarray
    eps: float
    nz: int
    dz: float
    z0: float
    layer_top: np.ndarray
    layer_vel: np.ndarray
    alpha: float
    cutoff: float
    snr_db: Optional[float] = None

    def summary(self) -> dict:
        d = {k: v for k, v in asdict(self).items() if not isinstance(v, np.ndarray)}
        d["nfreq"] = int(len(self.freq_hz))
        d["nlayer"] = int(len(self.layer_top))
        return d


def perturbation_blobs_3d(rng, nx, ny, dx, dy, nz, dz, z0, layer_top, layer_vel, nblob=3,
                          sigma=30.0, amp=0.05):
    """V(x, y, z) [ny][nx][nz] for Gaussian blobs of relative velocity change +-amp."""
    x = np.arange(nx) * dx
    y = np.arange(ny) * dy
    z = _depths(nz, dz, z0)
    c0 = velocity_at(z, layer_top, layer_vel)
    rel = np.zeros((ny, nx, nz))
    for b in range(nblob):
        xc = rng.uniform(0.15, 0.85) * nx * dx
        yc = rng.uniform(0.15, 0.85) * ny * dy
        zc = z0 + rng.uniform(0.2, 0.8) * nz * dz
        sgn = 1.0 if b % 2 == 0 else -1.0
        rel += sgn * amp * np.exp(-((y[:, None, None] - yc) ** 2 + (x[None, :, None] - xc) ** 2
                                    + (z[None, None, :] - zc) ** 2) / (2.0 * sigma ** 2))
    return _v_from_rel(rel, c0[None, None, :])


def perturbation_random_field_3d(rng, nx, ny, dx, dy, nz, dz, z0, layer_top, layer_vel,
                                 corr=40.0, rms=0.03):
    """V(x, y, z) [ny][nx][nz] for a Gaussian-correlated random relative velocity field."""
    white = rng.standard_normal((ny, nx, nz))
    ky = 2 * np.pi * np.fft.fftfreq(ny, dy)
    kx = 2 * np.pi * np.fft.fftfreq(nx, dx)
    kz = 2 * np.pi * np.fft.fftfreq(nz, dz)
    filt = np.exp(-0.25 * corr ** 2 * (ky[:, None, None] ** 2 + kx[None, :, None] ** 2
                                       + kz[None, None, :] ** 2))
    rel = np.real(np.fft.ifftn(np.fft.fftn(white) * filt))
    rel *= rms / max(np.sqrt(np.mean(rel ** 2)), 1e-300)
    z = _depths(nz, dz, z0)
    c0 = velocity_at(z, layer_top, layer_vel)
    return _v_from_rel(rel, c0[None, None, :])


def preset3d(name: str) -> Workload3D:
    """Finite-aperture workloads: ``small_3d`` (tests), ``line_fa`` (a 2D line with a
    finite aperture) and ``batched_3d`` (128 x 128 midpoints at 12.5 m, 16 x 16 half-offsets
    at 12.5 m (offsets every 25 m), 64 frequencies 4-50 Hz, 200 depths of 10 m, the 20-layer
    generator)."""
    if name == "small_3d":
        tops, vel = layers_gradient_staircase(1500.0, 3000.0, 120.0, 10.0, sub=2)
        return Workload3D(name, nx=16, ny=16, dx=10.0, dy=10.0, wx=4, wy=4,
                          freq_hz=freqs_uniform(4, 10.0, 40.0), eps=0.15, nz=12, dz=10.0,
                          z0=0.0, layer_top=tops, layer_vel=vel, alpha=1e-4, cutoff=1.0)
    if name == "line_fa":
        tops, vel = layers_gradient_staircase(1500.0, 3000.0, 320.0, 10.0, sub=2)
        return Workload3D(name, nx=64, ny=1, dx=10.0, dy=10.0, wx=16, wy=1,
                          freq_hz=freqs_uniform(12, 5.0, 40.0), eps=0.15, nz=32, dz=10.0,
                          z0=0.0, layer_top=tops, layer_vel=vel, alpha=1e-4, cutoff=1.0)
    if name == "batched_3d":
        tops, vel = layers_random(rng_for(2), 20, 2048.0)
        return Workload3D(name, nx=128, ny=128, dx=12.5, dy=12.5, wx=16, wy=16,
                          freq_hz=freqs_uniform(64, 4.0, 50.0), eps=0.15, nz=200, dz=10.0,
                          z0=0.0, layer_top=tops, layer_vel=vel, alpha=1e-2, cutoff=1.0)
    raise KeyError(name)
