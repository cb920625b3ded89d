"""Multi-GPU sharding of frame pairs.

Pairs are independent, so the path shards by whole pairs with no data exchange:
each rank tracks its own pairs on its own GPU. ``ShardedBatch`` is the runner: it
splits a batch's pair descriptors over the ranks by longest processing time and
tracks the rank's share through one ``BatchTracker``. Collectives are used only for
the timing (max over ranks) and the totals (sum over ranks) of a measurement.
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


def barrier() -> None:
    """Barrier of the default process group (nothing without one)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def reduce_scalar(value: float, op: str, device=None) -> float:
    """Sum or max of a scalar over the ranks of the default process group (the
    value itself when torch.distributed is not initialised)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def rank_and_world():
    """(rank, world size) of the default process group, or (0, 1) without one."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def shard_specs(specs, levels: int, radius: int, rank: int, world: int):
    """The batch indices and pair specs (W, H, win, step) of one rank's share."""
    costs = [pair_cost(W, H, win, step, levels, radius) for (W, H, win, step) in specs]
    idx = assign_pairs(costs, world)[rank]
    return idx, [tuple(specs[i]) for i in idx]


class ShardedBatch:
    """One rank's share of a batch of frame pairs of mixed sizes and steps.

    ``specs`` lists the whole batch's (W, H, win, step); every rank derives the same
    longest-processing-time split without communicating (``indices`` are this
    rank's batch indices, in increasing order) and tracks its pairs with a
    ``BatchTracker`` on its own device (created on first use). ``run`` takes the
    rank's own frames, in the order of ``indices``; results sit in ``tracker``'s
    per-pair outputs. A rank whose share is empty runs nothing.
    """

    def __init__(self, specs, params, device="cuda", rank: int | None = None, world: int | None = None,
                 lanes=0):
        r, w = rank_and_world()
        self.rank = r if rank is None else int(rank)
        self.world = w if world is None else int(world)
        if not 0 <= self.rank < self.world:
            raise ValueError("rank must lie in [0, world)")
        self.params, self.device, self.lanes = params, device, lanes
        self.indices, self.specs = shard_specs(specs, params.levels, params.radius, self.rank, self.world)
        self._tracker = None

    @property
    def tracker(self):
        if self._tracker is None and self.specs:
            from .api import BatchTracker
            self._tracker = BatchTracker(self.specs, self.params, self.device, self.lanes)
        return self._tracker

    @property
    def points(self) -> int:
        """Key-points of this rank's share."""
        return sum(((W - win) // step + 1) * ((H - win) // step + 1) for (W, H, win, step) in self.specs
                   if W >= win and H >= win)

    def run(self, frames1=None, frames2=None, use_graph: bool = True):
        """Tracks the rank's pairs (frames in the order of ``indices``; None after
        ``tracker.bind``)."""
        if self.tracker is not None:
            self.tracker.run(frames1, frames2, use_graph=use_graph)
        return self
