"""Partitioned solve of one survey line over ranks (one GPU per rank).

The midpoint-wavenumber subproblems are independent (Section "Two dimensions": eqs. DMV and M
decouple the wavenumbers k_m), but the data of one frequency feed every subproblem.  The
partition therefore shards the two axes differently:

* frequencies: contiguous shards of near-equal count; rank r holds D[f_r : f_{r+1}] and forms
  the split right-hand sides (eq. Split) of every subproblem at its frequencies;
* subproblems: contiguous ranges of near-equal cost (the Gram and the refinement are linear in
  a subproblem's rows, the factorisation is a fixed cost per subproblem); rank r solves m in
  [m_r, m_{r+1});
* one all-to-all moves the right-hand sides: a rank's exported rows are ordered by subproblem,
  so the rows that rank q owns form one contiguous block;
* each rank places the blocks it receives (one per source shard, by the source's frequency
  range), solves its subproblems, and the Vhat of all ranks (disjoint supports, zero outside
  each range) are summed by an all-reduce; every rank then holds V.

The kernel rows are not exchanged: every rank evaluates the Green's-function table of all
frequencies for its own subproblems.  The exchange is behind a small interface: ``Exchange``
over torch.distributed (batched point-to-point operations, which the gloo and nccl backends
both provide) and ``LocalGroup``, which runs every rank in sequence in one process.  The
per-rank compute is a backend; ``GpuBackend`` runs the library's kernels through the C ABI
(edt_row_offsets, edt_export_rhs, edt_import_rhs, edt_solve_imported, edt_inverse_vhat).

A backend provides ``sub_rows()`` (rows per subproblem of the whole job), ``shard(f0, f1)`` (an
object whose ``export(D_shard)`` returns (rows [R][2] complex tensor, offsets [nsub + 1])) and
``range(m0, m1)`` (an object with ``solve(blocks)``, blocks a list of (1-D real view of rows,
f_begin, f_end) in source order, returning Vhat [nsub][nz] complex128, and ``inverse(vhat)``).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


# ----------------------------------------------------------------------------- the plan
def plan_partition(sub_cost: Sequence[float], nfreq: int, world: int) -> Tuple[List[int], List[int]]:
    """(f_bounds, m_bounds), each world + 1 increasing boundaries: frequency shards of
    near-equal count, and contiguous non-empty subproblem ranges whose total costs are as equal
    as contiguity allows (boundary r at the prefix sum nearest to r / world of the total).
    ``sub_cost``: the cost of each subproblem (e.g. ``GpuBackend.sub_costs()``, or its rows)."""
    cost = np.asarray(sub_cost, dtype=np.float64)
    nsub = len(cost)
    if world < 1:
        raise ValueError("world must be positive")
    if world > nfreq or world > nsub:
        raise ValueError(f"{world} ranks need at least as many frequencies ({nfreq}) and "
                         f"subproblems ({nsub})")
    if np.any(cost < 0) or not np.all(np.isfinite(cost)):
        raise ValueError("costs must be finite and non-negative")
    f_bounds = [(nfreq * r) // world for r in range(world + 1)]
    cum = np.concatenate([[0.0], np.cumsum(cost)])
    total = cum[-1]
    m_bounds = [0]
    for r in range(1, world):
        target = total * r / world
        i = int(np.searchsorted(cum, target, side="left"))
        if i > 0 and (i > nsub or abs(cum[i - 1] - target) <= abs(cum[i] - target)):
            i -= 1
        # keep every range non-empty: at least one subproblem here and one per later rank
        i = min(max(i, m_bounds[-1] + 1), nsub - (world - r))
        m_bounds.append(i)
    m_bounds.append(nsub)
    return f_bounds, m_bounds


# ----------------------------------------------------------------------------- exchanges
class Exchange:
    """The collectives of one rank.  ``alltoallv(send)``: send[q] a 1-D tensor for rank q;
    returns recv, recv[s] the tensor rank s sent here.  ``allreduce_sum(t)``: sums t over the
    ranks, in place, and returns it."""
    rank: int = 0
    world: int = 1

    def alltoallv(self, send):
        raise NotImplementedError

    def allreduce_sum(self, t):
        raise NotImplementedError


class TorchDistExchange(Exchange):
    """Over torch.distributed (gloo with CPU tensors, nccl with CUDA tensors): the block sizes
    by an all-gather, then every send and receive in one batch."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def _global(self, r):
        return self.dist.get_global_rank(self.group, r) if self.group is not None else r

    def alltoallv(self, send):
        import torch
        dist = self.dist
        if len(send) != self.world:
            raise ValueError("one block per rank")
        dev, dtype = send[self.rank].device, send[self.rank].dtype
        sizes = torch.tensor([int(t.numel()) for t in send], dtype=torch.int64, device=dev)
        gathered = [torch.empty_like(sizes) for _ in range(self.world)]
        dist.all_gather(gathered, sizes, group=self.group)
        recv = [torch.empty(int(gathered[s][self.rank]), dtype=dtype, device=dev)
                for s in range(self.world)]
        recv[self.rank].copy_(send[self.rank])
        ops = []
        for q in range(self.world):
            if q == self.rank:
                continue
            if send[q].numel():
                ops.append(dist.P2POp(dist.isend, send[q].contiguous(), self._global(q), self.group))
            if recv[q].numel():
                ops.append(dist.P2POp(dist.irecv, recv[q], self._global(q), self.group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        return recv

    def allreduce_sum(self, t):
        import torch
        self.dist.all_reduce(torch.view_as_real(t) if t.is_complex() else t, group=self.group)
        return t


class LocalGroup:
    """Every rank in one process: the collectives over lists indexed by rank."""

    @staticmethod
    def alltoallv(sends):
        """sends[r][q] -> recvs[q][r]."""
        w = len(sends)
        return [[sends[r][q] for r in range(w)] for q in range(w)]

    @staticmethod
    def allreduce_sum(ts):
        total = ts[0].clone()
        for t in ts[1:]:
            total += t
        return [total.clone() for _ in ts]


# ----------------------------------------------------------------------------- the flow
def blocks_for_owners(rows, sub_off, m_bounds):
    """One rank's exported rows [R][2] (complex, ordered by subproblem) cut into the blocks of
    each owner's subproblem range, as flat real views (no copy)."""
    import torch
    flat = torch.view_as_real(rows)
    return [flat[int(sub_off[m_bounds[q]]):int(sub_off[m_bounds[q + 1]])].reshape(-1)
            for q in range(len(m_bounds) - 1)]


class PartitionedInversion:
    """One rank's share of the partitioned inversion; ``invert(D_shard)`` returns V on every
    rank.  The shard and range contexts are made once and reused by every call."""

    def __init__(self, backend, exchange: Exchange, f_bounds, m_bounds):
        r = exchange.rank
        if exchange.world != len(f_bounds) - 1 or exchange.world != len(m_bounds) - 1:
            raise ValueError("the plan's size differs from the group's")
        self.exchange, self.f_bounds, self.m_bounds = exchange, list(f_bounds), list(m_bounds)
        self.shard = backend.shard(f_bounds[r], f_bounds[r + 1])
        self.part = backend.range(m_bounds[r], m_bounds[r + 1])

    def invert(self, D_shard, out_dtype=None):
        ex, fb = self.exchange, self.f_bounds
        rows, sub_off = self.shard.export(D_shard)
        recv = ex.alltoallv(blocks_for_owners(rows, sub_off, self.m_bounds))
        vhat = self.part.solve([(recv[s], fb[s], fb[s + 1]) for s in range(ex.world)])
        ex.allreduce_sum(vhat)
        return self.part.inverse(vhat, out_dtype)


def invert_partitioned_local(backend, D, f_bounds, m_bounds, out_dtype=None):
    """Every rank of the partitioned inversion in sequence in this process: the steps of
    ``PartitionedInversion.invert`` with the collectives of ``LocalGroup``; returns V."""
    world = len(f_bounds) - 1
    shards = [backend.shard(f_bounds[r], f_bounds[r + 1]) for r in range(world)]
    parts = [backend.range(m_bounds[r], m_bounds[r + 1]) for r in range(world)]
    sends = []
    for r in range(world):
        rows, sub_off = shards[r].export(D[f_bounds[r]:f_bounds[r + 1]])
        sends.append(blocks_for_owners(rows, sub_off, m_bounds))
    recvs = LocalGroup.alltoallv(sends)
    vhats = [parts[r].solve([(recvs[r][s], f_bounds[s], f_bounds[s + 1]) for s in range(world)])
             for r in range(world)]
    return parts[0].inverse(LocalGroup.allreduce_sum(vhats)[0], out_dtype)


# ----------------------------------------------------------------------------- GPU backend
class GpuBackend:
    """Per-rank compute by the library on the current CUDA device and stream: a context over a
    frequency shard (export) and one over a subproblem range with every frequency (import,
    solve, inverse).  Line geometry only."""

    def __init__(self, cfg):
        from . import edt
        if cfg.geometry != edt.EDT_GEOM_LINE:
            raise ValueError("the partitioned solve is for the line geometry")
        self.cfg = cfg

    def sub_rows(self):
        """Solved rows per subproblem of the whole job, from a context without workspace."""
        from . import edt
        c, _arrays = self.cfg.c_config()
        ctx, _ = edt.edt_create(c)
        try:
            off = edt.edt_row_offsets(ctx, self.cfg.nx // 2 + 1)
        finally:
            edt.edt_destroy(ctx)
        return np.diff(off)

    # rows-equivalent of one factorisation per depth sample: the Gram and refinement cost about
    # 0.88 ns per row and the double-float Cholesky 3.8 us per subproblem on the 512-midpoint,
    # 256-depth, 128-frequency line (1.4 ms for 1.6 M rows, 0.98 ms for 257 factorisations);
    # a row costs O(nz^2) and a factorisation O(nz^3), so the ratio, 4350 at nz = 256, grows
    # with nz
    FACTOR_ROWS_PER_DEPTH = 17.0

    def sub_costs(self):
        """Per-subproblem cost in rows: its rows plus the rows-equivalent of its factorisation
        (none for a subproblem without rows)."""
        rows = self.sub_rows().astype(np.float64)
        return rows + np.where(rows > 0, self.FACTOR_ROWS_PER_DEPTH * self.cfg.nz, 0.0)

    def shard(self, f0, f1):
        import dataclasses
        return _GpuShard(dataclasses.replace(self.cfg, freq_hz=list(self.cfg.freq_hz)[f0:f1],
                                             sub_begin=0, sub_end=0))

    def range(self, m0, m1):
        import dataclasses
        if not m1 > m0:
            raise ValueError("a subproblem range must not be empty")
        return _GpuRange(dataclasses.replace(self.cfg, sub_begin=m0, sub_end=m1))


class _GpuShard:
    def __init__(self, cfg):
        from .edt import Solver
        self.s = Solver(cfg)

    def export(self, D_shard):
        import torch
        from . import edt
        s = self.s
        off = edt.edt_row_offsets(s.ctx, s.nsub)
        dt = torch.complex64 if s.cfg.precision == edt.EDT_MIXED else torch.complex128
        rows = torch.empty((int(off[-1]), 2), dtype=dt, device=s.device)
        edt.edt_export_rhs(s.ctx, D_shard.data_ptr(), s._cdtype(D_shard), rows.data_ptr(), s._stream())
        return rows, off


class _GpuRange:
    def __init__(self, cfg):
        from .edt import Solver
        self.s = Solver(cfg)

    def solve(self, blocks):
        import torch
        from . import edt
        s = self.s
        for blk, fb, fe in blocks:          # a row: (d_+, d_-), 4 reals
            edt.edt_import_rhs(s.ctx, blk.data_ptr() if blk.numel() else 0, blk.numel() // 4,
                               fb, fe, s._stream())
        vhat = torch.empty((s.nsub, s.cfg.nz), dtype=torch.complex128, device=s.device)
        edt.edt_solve_imported(s.ctx, vhat.data_ptr(), s._stream())
        return vhat

    def inverse(self, vhat, out_dtype=None):
        import torch
        from . import edt
        s = self.s
        V = torch.empty((s.cfg.nx, s.cfg.nz), dtype=out_dtype or torch.float64, device=s.device)
        edt.edt_inverse_vhat(s.ctx, vhat.data_ptr(), V.data_ptr(), s._rdtype(V), s._stream())
        return V
