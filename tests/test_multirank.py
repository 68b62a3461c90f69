"""Multi-rank host logic of bench.py on CPU ranks (gloo, world size 2).

Each rank inverts its own survey line (weak scaling, no collective on the data path); the
job's time is the maximum over ranks and the throughput counts every rank's subproblems.
"""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth
    t = bench.max_over_ranks(10.0 + 5.0 * rank, world)
    wl = synth.preset("small_2d")
    V = synth.perturbation_random_field(synth.rng_for(1, salt=bench.line_salt(rank)), wl.nx, wl.dx,
                                        wl.nz, wl.dz, wl.z0, wl.layer_top, wl.layer_vel)
    gathered = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, torch.tensor([float(V.sum())], dtype=torch.float64))
    out[rank] = (t, bench.job_throughput(world, 512, 10, t), [float(g) for g in gathered])
    dist.destroy_process_group()


def test_two_cpu_ranks_aggregate_like_the_bench():
    world = 2
    port = 29500 + (os.getpid() % 1000)
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, thr, sums = res[r]
        assert t == 15.0                                  # max over ranks
        assert thr == pytest.approx(world * 512 * 10 / 0.015)
        assert sums[0] != sums[1]                         # independent lines per rank


def test_single_rank_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_throughput(1, 512, 4, 2000.0) == pytest.approx(1024.0)
