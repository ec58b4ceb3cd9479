"""Environment sharding over ranks (one process per GPU).

Environments are independent (no coupling between them anywhere in the substep), so a
multi-GPU run is data parallel with no collective on the hot path: each rank owns a
contiguous range of environments and runs it on its own GPU.  The only collectives are
outside the step: the benchmark's barrier and max-over-ranks timing, and an optional gather
of per-environment results to one rank.
"""
from __future__ import annotations

from typing import Sequence


def shard_envs(costs: Sequence[float], world: int) -> list[tuple[int, int]]:
    """Contiguous (start, count) ranges of environments, one per rank, balancing the summed
    cost (particles x substeps x control steps) greedily in environment order.  Every
    environment lands in exactly one range; a rank can get none when there are fewer
    environments than ranks."""
    if world < 1:
        raise ValueError("world must be >= 1")
    n = len(costs)
    total = float(sum(costs))
    ranges = []
    start = 0
    acc = 0.0
    for r in range(world):
        if r == world - 1:
            end = n
        else:
            target = total * (r + 1) / world
            end = start
            # take environments while the running sum stays closer to the target with them
            while end < n - (world - 1 - r) and (acc + costs[end] <= target or
                                                 abs(acc + costs[end] - target) < abs(acc - target)):
                acc += costs[end]
                end += 1
        if r == world - 1:
            acc = total
        ranges.append((start, end - start))
        start = end
    return ranges


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar over the default process group (the value itself when no
    group is initialised)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """Sum of a per-rank scalar over the default process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
