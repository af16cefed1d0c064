"""Host logic of the multi-process path: one process per GPU, independent
problems per process (the batch's geometries are independent systems, so
they shard with no data-path collective), and the max-over-ranks time that
the benchmark reports.

Only torch.distributed plumbing is used here (a barrier and one all-reduce
of a scalar); no step of the solve crosses processes.
"""
from __future__ import annotations


def shard_by_cost(costs, world: int, rank: int):
    """Indices of the items of `costs` that rank `rank` of `world` solves.

    Longest-processing-time-first assignment: items in decreasing cost
    (ties by index) each go to the rank with the least assigned cost so far
    (ties by rank), so uneven geometries balance across GPUs. Every item goes
    to exactly one rank; the result is the same on every rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need world >= 1 and 0 <= rank < world")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    mine = []
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += float(costs[i])
        if r == rank:
            mine.append(i)
    return sorted(mine)


def reduce_max(value: float, device=None) -> float:
    """Max of `value` over all ranks of the default process group (the
    value itself when torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
