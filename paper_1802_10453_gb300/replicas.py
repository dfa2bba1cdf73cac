"""Host logic of runs on several GPUs (one process per GPU).

A single factorisation does not shard: its pivot chain is one global
sequence, so several GPUs run independent replicas.  A batch of independent
matrices shards by matrix, each rank factoring its own share with no
collective on the data path.  The one collective is the timing reduction:
the step time of a run is the maximum over the ranks, and the whole-job rate
is all ranks' work divided by it.
"""
from __future__ import annotations

import os


def dist_env():
    """(rank, world size, local rank) from the launcher's environment."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad RANK / WORLD_SIZE: %d / %d" % (rank, world))
    return rank, world, local


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The maximum of `value` over all ranks (all-reduce MAX of the default
    process group; the value itself when world == 1)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """All ranks' units of work per second of the slowest rank."""
    if seconds <= 0:
        raise ValueError("time must be positive")
    return float(units_per_rank) * world / seconds


def batch_shard(ns, rank: int, world: int):
    """Indices of the matrices of a batch (orders `ns`) that `rank` factors.

    Matrices are dealt in decreasing order of n^3 (the work of a full-rank
    factorisation; ties by index) to the rank holding the least work so far
    (ties to the lowest rank), so every matrix goes to exactly one rank and
    the work of two ranks differs by at most one matrix's.  Deterministic:
    every rank computes the same deal without communicating."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    order = sorted(range(len(ns)), key=lambda i: (-(max(int(ns[i]), 0) ** 3), i))
    load = [0] * world
    mine = []
    for i in order:
        w = min(range(world), key=lambda q: (load[q], q))
        load[w] += max(int(ns[i]), 0) ** 3
        if w == rank:
            mine.append(i)
    return sorted(mine)
