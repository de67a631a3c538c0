"""Multi-GPU execution: one process per GPU, independent work per process.

A single robust solve does not shard: the tile DAG's critical path (p + q - 1
dependent diagonal solves) and its cross-tile updates would need a point-to-point
exchange of Y tiles after every diagonal solve.  So N GPUs run N independent solves
(replicas), or split a batch of independent equations between them.  The only
exchange is host-side: the slowest rank's time (a MAX reduction) and, for a split
batch, each rank's share of the equations.
"""
from __future__ import annotations

import heapq


def lpt_shards(costs, world_size: int) -> list[list[int]]:
    """Split independent units over ``world_size`` ranks, longest processing time
    first: units in decreasing cost, each to the rank with the least total so far
    (ties to the lower rank, so every rank computes the same split).  Returns each
    rank's unit indices in increasing order."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(world_size)]
    shards: list[list[int]] = [[] for _ in range(world_size)]
    for i in order:
        load, r = heapq.heappop(heap)
        shards[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(s) for s in shards]


def max_over_ranks(value: float) -> float:
    """The largest ``value`` over all ranks (the rank's own value when no process group
    is running).  The reduction runs on the process group's device (CUDA for NCCL)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world_size: int, slowest_seconds: float) -> float:
    """Units per second of the whole job: every rank's units over the slowest rank's
    time (weak scaling: each rank does the same amount of work)."""
    return world_size * units_per_rank / slowest_seconds
