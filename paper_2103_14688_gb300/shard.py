"""Host-side logic of the multi-GPU path: independent queries sharded across
ranks, no collective on the data path.

Index creation of different queries shares nothing, so N GPUs run N disjoint
sets of queries (weak scaling: the per-rank work is fixed).  The only
collectives are outside the data path: a barrier, the maximum of the ranks'
timed totals, and gathering per-query summaries on rank 0.
"""
from __future__ import annotations

from typing import Callable, List, Sequence, Tuple


def rank_seed(base: int, rank: int) -> int:
    """Seed of the query a rank generates (distinct per rank)."""
    return int(base) + int(rank)


def partition(costs: Sequence[float], world: int) -> List[List[int]]:
    """Longest-processing-time assignment of query indices to ranks: queries
    by decreasing cost, each to the least-loaded rank.  Every index appears
    exactly once; ranks keep their indices in increasing order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0.0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: (-float(costs[k]), k)):
        r = min(range(world), key=lambda j: (load[j], j))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def query_cost(n: int, n_states: int) -> float:
    """Cost proxy of one query: bits of its dense state blocks, n^2 |Q|."""
    return float(n) * float(n) * float(n_states)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of a per-rank float over the process group (identity without one)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_results(local: Sequence[Tuple[int, object]], n_total: int, dist=None) -> List[object]:
    """Collect (index, result) pairs of every rank into one list ordered by
    query index (on every rank)."""
    if dist is None:
        out = [None] * n_total
        for i, v in local:
            out[i] = v
        return out
    world = dist.get_world_size()
    parts = [None] * world
    dist.all_gather_object(parts, list(local))
    out = [None] * n_total
    for p in parts:
        for i, v in p:
            out[i] = v
    return out


def run_sharded(costs: Sequence[float], rank: int, world: int, runner: Callable[[List[int]], List[object]],
                dist=None) -> List[object]:
    """Run this rank's share of the queries and return every query's result
    (ordered by index) on every rank."""
    mine = partition(costs, world)[rank]
    res = runner(mine) if mine else []
    return gather_results(list(zip(mine, res)), len(costs), dist)
