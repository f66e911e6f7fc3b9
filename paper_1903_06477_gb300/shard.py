"""Instance sharding of batched solves across GPUs, one process per GPU.

The instances of a batch are independent problems, so a batch splits across
ranks with no exchange on the data path: every rank solves its share with its
own scs_batch on its own GPU, and only the per-instance results cross ranks,
once, after the solves.  The split balances work by the cost of one outer
iteration of an instance, which is proportional to nnz(A) + n + m (the sparse
products and the vector passes), with the longest-processing-time rule:
instances by decreasing cost, each given to the rank with the least total so
far (ties to the lower rank, equal costs in index order).  The rule is
deterministic, so every rank computes the same partition from the same
instance list without communicating.  Host logic only.
"""
from __future__ import annotations

import heapq


def instance_cost(prob) -> int:
    """nnz(A) + n + m of one instance (dict with a scipy.sparse 'A')."""
    A = prob["A"]
    return int(A.nnz) + int(A.shape[0]) + int(A.shape[1])


def partition(costs, world: int):
    """Instance indices of each rank: list of `world` sorted lists covering
    range(len(costs)) exactly once, balanced by the longest-processing-time
    rule on `costs`."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(p) for p in parts]


def loads(costs, parts):
    return [sum(costs[i] for i in p) for p in parts]


def gather(local_idx, local_results, total: int, dist=None):
    """Every rank's results in global instance order, on every rank.
    local_results[k] belongs to instance local_idx[k]; results are any
    picklable objects (per-instance status, iterations, objective ...)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        pieces = [(list(local_idx), list(local_results))]
    else:
        pieces = [None] * dist.get_world_size()
        dist.all_gather_object(pieces, (list(local_idx), list(local_results)))
    out = [None] * total
    seen = 0
    for idx, res in pieces:
        if len(idx) != len(res):
            raise ValueError("indices and results differ in length")
        for i, r in zip(idx, res):
            if out[i] is not None:
                raise ValueError(f"instance {i} reported twice")
            out[i] = r
            seen += 1
    if seen != total:
        raise ValueError(f"{total - seen} instances missing from the gather")
    return out
