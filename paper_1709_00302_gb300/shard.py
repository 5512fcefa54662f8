"""Partition of a batch of independent band reductions over ranks (one process per GPU).

The reductions of a batch share nothing, so several GPUs split the matrices between them
and exchange no data: each rank reduces its own share with the batched entry points, and
only the timings and the device status words meet on the host.  The split is greedy
longest-processing-time first on the nominal flop counts of the two reductions (Section
2.1: 4n^3/3 for sy2sb; Section 3.1: 4(mn^2 - n^3/3) for ge2gb).  It is deterministic, so
every rank computes the same partition without talking to the others.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


def sy2sb_flops(n: int) -> float:
    """Nominal flops of sy2sb on an n x n matrix (Section 2.1)."""
    return 4.0 * n ** 3 / 3.0


def ge2gb_flops(m: int, n: int) -> float:
    """Nominal flops of ge2gb on an m x n matrix, m >= n (Section 3.1)."""
    return 4.0 * (m * n * n - n ** 3 / 3.0)


def shard_lpt(costs: Sequence[float], world: int) -> Tuple[List[List[int]], List[float]]:
    """Greedy LPT: the items, in decreasing cost (ties by index), each go to the rank with
    the smallest load so far (ties to the lowest rank).  Returns, per rank, the sorted
    indices it owns and its total cost.  The largest load exceeds the smallest by at most
    the largest single cost, and is within 4/3 of the best possible."""
    if world < 1:
        raise ValueError("world must be >= 1")
    loads = [0.0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda q: (-float(costs[q]), q)):
        r = min(range(world), key=lambda q: (loads[q], q))
        parts[r].append(i)
        loads[r] += float(costs[i])
    return [sorted(p) for p in parts], loads


def batched_shard(sym: Sequence[Tuple[int, int]], gen: Sequence[Tuple[int, int, int]], world: int,
                  rank: int) -> Tuple[List[int], List[int]]:
    """This rank's share of a mixed batch: the indices of its symmetric matrices (shapes
    (n, w)) and of its general ones (shapes (m, n, w)), both kinds balanced together."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    costs = [sy2sb_flops(n) for n, _ in sym] + [ge2gb_flops(m, n) for m, n, _ in gen]
    parts, _ = shard_lpt(costs, world)
    mine = parts[rank]
    ns = len(sym)
    return [i for i in mine if i < ns], [i - ns for i in mine if i >= ns]
