"""Sharding independent instances over ranks (one GPU per rank) for the batched and served
forms.  A single bisection does not shard (its matching and contraction exchange data every
pass), but independent instances do: every rank partitions its own share, with no collective on
the data path; only the final timing is reduced (maximum over ranks).

The assignment is longest-processing-time first: instances sorted by cost (descending, ties by
index) go to the rank with the smallest load so far (ties to the lower rank), so every rank
computes the same assignment from the same costs without communicating.
"""
from __future__ import annotations

import heapq


def assign(costs, world: int):
    """Returns `world` lists of instance indices (ascending within each list)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(x) for x in out]


def my_share(costs, rank: int, world: int):
    return assign(costs, world)[rank]


def serve_share(costs, arrivals, rank: int, world: int):
    """The served form's share of a request trace: this rank's longest-processing-time share of
    the requests, in arrival order, with their arrival times.  Every rank serves its share with its
    own server on its own GPU; nothing is exchanged while serving."""
    mine = sorted(my_share(costs, rank, world), key=lambda i: (arrivals[i], i))
    return mine, [arrivals[i] for i in mine]


def min_over_ranks(value: float) -> float:
    """Minimum of a float over the default process group (identity without one)."""
    return -max_over_ranks(-float(value))


def max_over_ranks(value: float) -> float:
    """Maximum of a float over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
