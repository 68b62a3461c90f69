"""Helpers shared by the GPU parity tests (CUDA path through the C ABI vs the oracle)."""
import numpy as np

import synth


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def small_workload(nx=32, nz=24, nf=6, fmin=5.0, fmax=40.0, dx=10.0, dz=10.0, z0=0.0,
                   alpha=1e-5, cutoff=1.0, layers=None, eps=0.15):
    if layers is None:
        layers = synth.layers_gradient_staircase(1500.0, 3000.0, nz * dz, dz, sub=2)
    tops, vel = layers
    return synth.Workload("test", nx=nx, dx=dx, freq_hz=synth.freqs_uniform(nf, fmin, fmax),
                          eps=eps, nz=nz, dz=dz, z0=z0, layer_top=np.asarray(tops),
                          layer_vel=np.asarray(vel), alpha=alpha, cutoff=cutoff)


def blobs(wl, salt=0):
    rng = synth.rng_for(0, salt=salt)
    return synth.perturbation_blobs(rng, wl.nx, wl.dx, wl.nz, wl.dz, wl.z0, wl.layer_top,
                                    wl.layer_vel, nblob=3, sigma=30.0, amp=0.05)


def dev(a):
    """A contiguous CUDA tensor copy of a numpy array."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()
