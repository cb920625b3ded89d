"""Multi-GPU sharding of frame pairs (host logic only).

Pairs are independent, so the path shards by whole pairs with no data exchange:
each rank tracks its own pairs on its own GPU. Collectives are used only for the
timing (max over ranks) and the totals (sum over ranks) of a measurement.
"""
from __future__ import annotations

import torch


def pair_cost(W: int, H: int, win: int, step: int, levels: int, radius: int) -> int:
    """Work proxy of one pair: key-points x levels x support samples."""
    if W < win or H < win:
        return 0
    n = ((W - win) // step + 1) * ((H - win) // step + 1)
    return n * levels * (2 * radius + 1) ** 2


def assign_pairs(costs, world: int):
    """Longest-processing-time assignment of pair indices to `world` ranks.

    Deterministic (ties break by index), so every rank computes the same split
    without communicating. Returns one sorted index list per rank.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    loads = [0] * world
    shards = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        r = min(range(world), key=lambda k: (loads[k], k))
        shards[r].append(i)
        loads[r] += costs[i]
    return [sorted(s) for s in shards]


def reduce_scalar(value: float, op: str, device=None) -> float:
    """Sum or max of a scalar over the ranks of the default process group (the
    value itself when torch.distributed is not initialised)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())
