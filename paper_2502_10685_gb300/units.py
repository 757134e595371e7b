"""Distribution of independent units over the ranks of a job (one process per
GPU).  A unit -- a circuit of a batch, a parameter-shift copy, a serving
request -- needs no data from any other (each stabilizer generator and each
circuit is propagated on its own, Sec. IV-B), so ranks share no collective on
the data path: the host assigns units, every rank runs its share, and the
results are gathered to one rank at the end.

Costs are coefficient updates, vectors x gates x 4^n, the work one unit puts
on a GPU.
"""
from __future__ import annotations

import heapq
from typing import Any, List, Optional, Sequence, Tuple


def unit_cost(n: int, m: int, vectors: int = 1) -> int:
    """Coefficient updates of `vectors` vectors of 4^n entries through m gates."""
    return int(vectors) * int(m) * 4 ** int(n)


def lpt_partition(costs: Sequence[float], world: int) -> List[List[int]]:
    """Longest processing time first: items in order of decreasing cost (ties
    by index) each go to the rank with the least assigned cost so far (ties to
    the lower rank).  Returns, per rank, its item indices in ascending order.
    Deterministic, every index exactly once; the largest load is at most the
    mean load plus the largest single cost."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap: List[Tuple[float, int]] = [(0.0, r) for r in range(world)]
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(p) for p in parts]


def route_in_arrival_order(costs: Sequence[float], world: int) -> List[int]:
    """Serving: the rank of each request, taken in arrival order, to the rank
    with the least work assigned so far (ties to the lower rank).  A pure
    function of the cost sequence, so every rank computes the same routing
    without exchanging anything."""
    if world < 1:
        raise ValueError("world must be >= 1")
    heap: List[Tuple[float, int]] = [(0.0, r) for r in range(world)]
    out = []
    for c in costs:
        load, r = heapq.heappop(heap)
        out.append(r)
        heapq.heappush(heap, (load + float(c), r))
    return out


def gather_to_root(local_indices: Sequence[int], local_results: Sequence[Any], n_total: int,
                   dist=None, root: int = 0) -> Optional[List[Any]]:
    """Every rank's results, placed at their item indices, on `root` (None on
    the other ranks).  Without a process group (or with one rank) the local
    results are the whole set."""
    if len(local_indices) != len(local_results):
        raise ValueError("one result per index")
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        pieces = [(list(local_indices), list(local_results))]
        rank = root
    else:
        pieces = [None] * dist.get_world_size()
        dist.all_gather_object(pieces, (list(local_indices), list(local_results)))
        rank = dist.get_rank()
    if rank != root:
        return None
    out: List[Any] = [None] * n_total
    filled = [False] * n_total
    for idx, res in pieces:
        for i, r in zip(idx, res):
            if filled[i]:
                raise ValueError("item %d returned twice" % i)
            out[i] = r
            filled[i] = True
    if not all(filled):
        raise ValueError("%d of %d items returned" % (sum(filled), n_total))
    return out
