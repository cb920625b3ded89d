"""Multi-rank host logic of the sharded path on CPU (gloo, world size 2): every
rank derives the same split of the 64-pair batch (in the ShardedBatch runner as in
assign_pairs), the shards cover each pair once and are balanced, the timing and
total reductions agree, and a rank that leaves makes the other's next collective
fail within its timeout instead of hanging."""
import datetime
import os
import socket

import pytest
import torch.multiprocessing as mp

import synth
from paper_1901_09971_gb300 import shard


def batch_costs():
    specs = synth.make_batch_specs(64, 3000)
    return [shard.pair_cost(W, H, 8, step, 3, 4) for (W, H, step) in specs]


def test_assignment_covers_every_pair_once_and_balances():
    costs = batch_costs()
    for world in (1, 2, 4, 8):
        shards = shard.assign_pairs(costs, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in s) for s in shards]
        assert max(loads) - min(loads) <= max(costs)  # LPT bound
    assert shard.assign_pairs(costs, 2) == shard.assign_pairs(list(costs), 2)  # deterministic
    with pytest.raises(ValueError):
        shard.assign_pairs(costs, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, mode, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    costs = batch_costs()
    mine = shard.assign_pairs(costs, world)[rank]
    if mode == "ok":
        # the runner's share is the same split, derived from the process group
        from paper_1901_09971_gb300 import RlofParams
        specs = [(W, H, 8, step) for (W, H, step) in synth.make_batch_specs(64, 3000)]
        runner = shard.ShardedBatch(specs, RlofParams(levels=3, radius=4), device="cpu")
        assert (runner.rank, runner.world) == (rank, world) and runner.indices == mine
        assert runner.specs == [specs[i] for i in mine]
        total = shard.reduce_scalar(sum(costs[i] for i in mine), "sum")
        points = shard.reduce_scalar(runner.points, "sum")
        slowest = shard.reduce_scalar(1.0 + rank, "max")
        out.put((rank, mine, total, slowest, points))
        dist.barrier()
        dist.destroy_process_group()
    else:  # rank 1 leaves between steps; rank 0's next collective must fail, not hang
        if rank == 1:
            out.put((rank, "left"))
            return
        try:
            shard.reduce_scalar(1.0, "sum")
            out.put((rank, "no error"))
        except Exception as e:  # noqa: BLE001 - any collective error is the expected outcome
            out.put((rank, "error", type(e).__name__))


def _run(mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    return sorted(res, key=lambda r: r[0])


def test_two_ranks_split_and_reduce():
    """Both ranks' runners derive the split from the process group; their shares
    cover the 64-pair batch once, and the reduced totals (work, key-points, the
    slowest rank's time) agree."""
    res = _run("ok")
    costs = batch_costs()
    (r0, m0, t0, s0, p0), (r1, m1, t1, s1, p1) = res
    assert sorted(m0 + m1) == list(range(len(costs))) and not set(m0) & set(m1)
    assert t0 == t1 == float(sum(costs))
    assert s0 == s1 == 2.0
    specs = synth.make_batch_specs(64, 3000)
    assert p0 == p1 == float(sum(((W - 8) // st + 1) * ((H - 8) // st + 1) for (W, H, st) in specs))


def test_runner_without_a_process_group_takes_the_whole_batch():
    from paper_1901_09971_gb300 import RlofParams
    specs = [(W, H, 8, step) for (W, H, step) in synth.make_batch_specs(64, 3000)]
    runner = shard.ShardedBatch(specs, RlofParams(levels=3, radius=4), device="cpu")
    assert (runner.rank, runner.world) == (0, 1) and runner.indices == list(range(64))
    shares = [shard.ShardedBatch(specs, RlofParams(levels=3, radius=4), device="cpu", rank=r, world=8) for r in range(8)]
    assert sorted(i for sh in shares for i in sh.indices) == list(range(64))
    with pytest.raises(ValueError):
        shard.ShardedBatch(specs, RlofParams(levels=3, radius=4), rank=2, world=2)


def test_departed_rank_fails_collective_instead_of_hanging():
    res = _run("leave")
    assert res[1] == (1, "left")
    assert res[0][1] == "error"
