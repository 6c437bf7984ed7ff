"""Multi-GPU bookkeeping for replica runs.

The tiled factorization of one matrix does not shard without a 2-D tile
distribution and per-step panel broadcasts, so several GPUs run independent
problems: each rank factors its own matrix (or its own share of a batch) on
its own GPU, with no collective on the data path.  Only timing and counting
cross ranks: the job time is the maximum over ranks and the job rate is the
work of all ranks divided by it (weak scaling).
"""
from __future__ import annotations

import torch


def max_over_ranks(t: float, dist=None, device=None) -> float:
    """The maximum of a per-rank time over all ranks (identity without dist)."""
    if dist is None or not dist.is_initialized():
        return float(t)
    x = torch.tensor([float(t)], dtype=torch.float64, device=device)
    dist.all_reduce(x, op=dist.ReduceOp.MAX)
    return float(x.item())


def job_rate(units_per_rank, t_max: float) -> float:
    """Whole-job throughput: the units of every rank over the slowest rank's time."""
    return float(sum(units_per_rank)) / t_max


def shard_batch(costs, world: int):
    """Split a batch of independent problems over `world` ranks so that the
    ranks' total costs are as even as a greedy longest-first assignment makes
    them.  Returns one sorted index list per rank (every index exactly once)."""
    order = sorted(range(len(costs)), key=lambda b: -costs[b])
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for b in order:
        r = min(range(world), key=lambda x: load[x])
        parts[r].append(b)
        load[r] += costs[b]
    return [sorted(p) for p in parts]
