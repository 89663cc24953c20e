"""Spreading one batch of SF instances over ranks (one process per GPU).

Instances are independent: T couples nothing across them, so a multi-GPU solve is a
partition of the batch with no collective on the data path.  The per-instance cost
of an iteration is dominated by its rows: P H pair rows (P = n (n - 1) / 2) and
n n_obs H obstacle rows.  ``balance`` assigns instances to ranks by that cost, largest
first, each to the least-loaded rank (ties to the lower rank), which is deterministic
so that every rank computes the same partition without communicating.
``gather`` brings per-rank results back into batch order on every rank.
"""
from __future__ import annotations


def instance_cost(inst) -> int:
    """Rows per iteration: P H robot-pair rows plus n n_obs H obstacle rows (plus the
    n H box rows, so that an instance without partners still costs something)."""
    n, n_obs, H = int(inst["n"]), int(inst["n_obs"]), int(inst["H"])
    return (n * (n - 1) // 2) * H + n * n_obs * H + n * H


def balance(costs, world: int):
    """Greedy longest-first partition of instance indices over ``world`` ranks; returns
    one ascending index list per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda k: (-costs[k], k))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(k)
        load[r] += costs[k]
    return [sorted(p) for p in parts]


def shard(insts, rank: int, world: int):
    """This rank's share: (batch indices, instances)."""
    idx = balance([instance_cost(i) for i in insts], world)[rank]
    return idx, [insts[k] for k in idx]


def gather(local, idx, world: int, group=None):
    """Every rank's ``local`` results (one per index in ``idx``) back in batch order, on
    every rank (``torch.distributed.all_gather_object``; host objects)."""
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, (list(idx), list(local)), group=group)
    n = sum(len(p[0]) for p in parts)
    out = [None] * n
    for ids, vals in parts:
        for k, v in zip(ids, vals):
            out[k] = v
    return out


def max_over_ranks(x: float, device="cpu", group=None) -> float:
    """The maximum of a host scalar over all ranks (the step time of a job is its slowest
    rank's)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
