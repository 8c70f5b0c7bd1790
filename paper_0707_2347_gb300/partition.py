"""Host-side sharding of a batch of independent products across ranks.

The batched workload (many C <- A B + C problems of uneven shapes) has no
exchange step: every problem is independent, so ranks split the problems and
run them with no data-path collective.  Problems are assigned by
longest-processing-time-first on the library's modelled cost
(swmm_autotune), which keeps the ranks' totals within the largest single
problem of each other.
"""
from __future__ import annotations

import heapq

from . import swmm as S


def modelled_cost(shape, mode=S.MODP, p=65521) -> float:
    m, k, n = shape
    return S.autotune(m, k, n, mode, p)[2]


def assign(shapes, world: int, modes=None, p=65521):
    """List of problem-index lists, one per rank (deterministic)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    modes = modes or [S.MODP] * len(shapes)
    cost = [modelled_cost(s, md, p) for s, md in zip(shapes, modes)]
    order = sorted(range(len(shapes)), key=lambda i: (-cost[i], i))
    heap = [(0.0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + cost[i], r))
    return [sorted(x) for x in out], cost
