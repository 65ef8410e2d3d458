"""Sharding of independent slabs across ranks (one process per GPU).

A batch of independent slabs needs no exchange while it advances: each rank
runs its share as one batched context, and only per-slab results (moments,
totals) are gathered at the end.  Shares come from the greedy
longest-processing-time rule (Graham 1969): slabs sorted by cost
(nodes x velocities x steps) go one by one to the currently least-loaded
rank, which keeps the largest load within 4/3 of the optimum.
"""
from __future__ import annotations

import heapq


def lpt_partition(costs, world: int):
    """Returns `world` lists of slab indices (each in ascending index order)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(p) for p in parts]


def slab_costs(slabs, steps: int = 1):
    """Cost of each slab dict {nz, Q, ...}: node-velocity updates over `steps`."""
    return [s["nz"] * s["Q"] * steps for s in slabs]


def my_share(slabs, rank: int, world: int, steps: int = 1):
    """Indices of the slabs rank `rank` advances."""
    return lpt_partition(slab_costs(slabs, steps), world)[rank]


def gather_by_slab(local: dict, nslab: int, group=None):
    """Gathers {slab index: result} from every rank (torch.distributed, any
    backend) and returns the list of results in slab order on every rank."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    everything = [None] * world
    dist.all_gather_object(everything, local, group=group)
    out = [None] * nslab
    for part in everything:
        for i, v in part.items():
            if out[i] is not None:
                raise RuntimeError(f"slab {i} reported by two ranks")
            out[i] = v
    missing = [i for i, v in enumerate(out) if v is None]
    if missing:
        raise RuntimeError(f"slabs {missing[:8]} reported by no rank")
    return out
