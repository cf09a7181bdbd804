"""Instance sharding across GPUs (one process per GPU).

Independent solves (a mesh and a source) share nothing, so a batch is split across
ranks with no exchange during the solve; results are gathered on rank 0 at the end.
A single solve is not split: partitioning a mesh would need an all-to-all of windows
crossing the cut every iteration, which the method does not have.
"""
from __future__ import annotations

import heapq
from typing import Callable, Sequence


def shard_instances(weights: Sequence[float], world_size: int) -> list[list[int]]:
    """Longest-processing-time split of instances over ranks, balanced by weight
    (e.g. face count).  Deterministic: ties go to the lower rank / lower index."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(len(weights)), key=lambda i: (-float(weights[i]), i))
    heap = [(0.0, r) for r in range(world_size)]
    out = [[] for _ in range(world_size)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + float(weights[i]), r))
    for lst in out:
        lst.sort()
    return out


def solve_sharded(n_instances: int, weights: Sequence[float], solve_fn: Callable[[list[int]], list],
                  rank: int, world_size: int, group=None):
    """Run `solve_fn(indices)` on this rank's shard and gather every instance's result
    on rank 0 (other ranks get None).  Uses torch.distributed object collectives, so
    any backend works (gloo on CPU, nccl on GPUs)."""
    shards = shard_instances(weights, world_size)
    mine = shards[rank]
    local = solve_fn(mine) if mine else []
    if world_size == 1:
        return list(local)
    import torch.distributed as dist
    payload = list(zip(mine, local))
    gathered = [None] * world_size if rank == 0 else None
    dist.gather_object(payload, gathered, dst=0, group=group)
    if rank != 0:
        return None
    res = [None] * n_instances
    for part in gathered:
        for i, r in part:
            res[i] = r
    return res
