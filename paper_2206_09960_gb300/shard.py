"""Row sharding of the Power-psi iteration over ranks, and the reductions of a multi-rank run.

The iteration of Eq. 14 pulls, for every leader row i, the gathered values u_j = s_j/sigma_j
of its followers j.  Split the rows into contiguous ranges balanced by their nonzeros (plus a
per-row cost for the epilogue); every rank then computes y, s and u for its own rows, and
one exchange step per iteration makes the new u whole again on every rank (an allgather of
the ranks' row ranges) while the L1 gap of Eq. 15 is the sum of the ranks' partial gaps (an
allreduce).  Independent problems (replicas, scenario batches, independent graphs) need no
exchange at all; their only multi-rank step is the timing reduction (the maximum over
ranks of the per-step time).

Everything here is host logic on ``torch.distributed`` (gloo for CPU tensors, NCCL for CUDA
tensors); the per-rank arithmetic is the caller's.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def partition_rows(row_ptr, world: int, row_cost: int = 1) -> np.ndarray:
    """Contiguous row ranges balanced by work: rank r owns rows [bounds[r], bounds[r+1]).

    The work of row i is its nonzeros plus ``row_cost``; the cuts are the rows where the
    running work first reaches r/world of the total, so every range holds at most one row's
    work more than its share.  ``row_ptr`` has n_rows + 1 entries."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    n_rows = row_ptr.size - 1
    if world < 1:
        raise ValueError("world must be >= 1")
    if n_rows < 0:
        raise ValueError("row_ptr needs at least one entry")
    work = np.diff(row_ptr) + int(row_cost)
    cum = np.concatenate([[0], np.cumsum(work)])
    total = int(cum[-1])
    targets = (np.arange(1, world, dtype=np.int64) * total) // world
    cuts = np.searchsorted(cum, targets, side="left")
    bounds = np.concatenate([[0], np.clip(cuts, 0, n_rows), [n_rows]]).astype(np.int64)
    return np.maximum.accumulate(bounds)


@dataclass(frozen=True)
class ShardPlan:
    """The row ranges of every rank and the layout of the exchange."""

    bounds: np.ndarray  # [world + 1]
    rank: int

    @property
    def world(self) -> int:
        return int(self.bounds.size - 1)

    @property
    def rows(self) -> tuple[int, int]:
        return int(self.bounds[self.rank]), int(self.bounds[self.rank + 1])

    def counts(self) -> np.ndarray:
        return np.diff(self.bounds)


def make_plan(row_ptr, world: int, rank: int, row_cost: int = 1) -> ShardPlan:
    if not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    return ShardPlan(partition_rows(row_ptr, world, row_cost), rank)


def allgather_rows(local, plan: ShardPlan, group=None):
    """Every rank's values for its own rows -> the whole vector, on every rank.

    ``local`` is a 1-D torch tensor with plan.counts()[rank] entries (CPU for gloo, CUDA for
    NCCL).  The ranges are padded to the longest one for the collective and cut back."""
    import torch
    import torch.distributed as dist

    counts = plan.counts()
    if local.numel() != counts[plan.rank]:
        raise ValueError("local holds %d values, the plan gives this rank %d" % (local.numel(), counts[plan.rank]))
    width = int(counts.max()) if counts.size else 0
    padded = torch.zeros(width, dtype=local.dtype, device=local.device)
    padded[: local.numel()] = local
    parts = [torch.empty_like(padded) for _ in range(plan.world)]
    dist.all_gather(parts, padded, group=group)
    return torch.cat([p[: int(c)] for p, c in zip(parts, counts)])


def allreduce_sum(x: float, device="cpu", group=None) -> float:
    """Sum of one FP64 scalar over ranks (the L1 gap of Eq. 15 from the ranks' partial sums)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())


def max_over_ranks(x: float, device="cpu", group=None) -> float:
    """Maximum of one scalar over ranks (the time of a step of the whole job)."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
