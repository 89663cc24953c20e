"""Multi-rank host logic, on CPU with world-size-2 gloo process groups.

Each rank takes its balanced share of an uneven batch, computes a host stand-in of a
per-instance result, and gathers everyone's results back in batch order; the step time
of the job is the max over ranks; bench.py's weak-scaling workloads differ per rank."""
import os
import socket

import numpy as np
import pytest

import sfgen
from paper_2510_09204_b300 import shard

WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world)
        insts = sfgen.make_batch(3, B=12)
        idx, mine = shard.shard(insts, rank, world)
        local = [float(np.asarray(i["xi"]).sum()) for i in mine]
        gathered = shard.gather(local, idx, world)
        t = shard.max_over_ranks(1.0 + rank)
        import bench
        _, b, pairs, _ = bench.workload(1, rank)
        seeds = [None] * world
        dist.all_gather_object(seeds, float(np.asarray(b[0]["xi"]).sum()))
        dist.destroy_process_group()
        q.put((rank, idx, gathered, t, seeds, pairs, None))
    except Exception as e:  # reported to the parent, never swallowed
        q.put((rank, None, None, None, None, None, repr(e)))


def test_two_rank_sharding_gather_and_timing():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, WORLD, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(WORLD):
        r = q.get(timeout=240)
        res[r[0]] = r
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(WORLD):
        assert res[r][6] is None, res[r][6]
    insts = sfgen.make_batch(3, B=12)
    want = [float(np.asarray(i["xi"]).sum()) for i in insts]
    idx = [res[r][1] for r in range(WORLD)]
    assert sorted(idx[0] + idx[1]) == list(range(len(insts)))        # a partition
    assert not set(idx[0]) & set(idx[1])
    for r in range(WORLD):
        assert res[r][2] == want                                     # batch order on every rank
        assert res[r][3] == 2.0                                      # max over ranks
    costs = [shard.instance_cost(i) for i in insts]
    loads = [sum(costs[k] for k in p) for p in idx]
    assert max(loads) - min(loads) <= max(costs)                     # greedy balance bound
    s0 = res[0][4]
    assert s0[0] != s0[1]                                            # distinct weak-scaling batches
    assert res[0][5] == res[1][5]                                    # same shape of work per rank


def test_balance_is_deterministic_and_complete():
    costs = [5, 9, 1, 9, 3, 7, 2, 2]
    p3 = shard.balance(costs, 3)
    assert p3 == shard.balance(list(costs), 3)
    assert sorted(sum(p3, [])) == list(range(len(costs)))
    assert shard.balance(costs, 1) == [list(range(len(costs)))]
    with pytest.raises(ValueError):
        shard.balance(costs, 0)
