"""Host-side logic of the multi-GPU paths.

Independent queries.  Index creation of different queries shares nothing,
so N GPUs run N disjoint sets of queries (weak scaling: the per-rank work is
fixed).  The only collectives are outside the data path: a barrier, the
maximum of the ranks' timed totals, and gathering per-query summaries.

One query over several GPUs (the multi-GPU version Sec. 6 leaves as future
work), split by the columns of the closure.  Row x of a closure block
C[s,t] is the OR, over the product edges (s,x) -> (u,y), of row y of C[u,t]
(and of bit y itself when u = t); restricted to a range of columns (target
vertices) it needs only the same columns of the rows it reads.  So every rank
keeps the whole graph and the whole M2, computes C3 on its own column range,
and extracts the new edges that fall in its columns.  The only exchange is
one all-gather per iteration of Listing 1: every rank's new edges (its
columns of A2), which together form the next iteration's A2 on every rank.
The loop ends after the first iteration in which no rank found an edge,
which is the unsharded loop's last iteration too.
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


# ---------------------------------------------------------------------------
# One query split over ranks by closure columns.
# ---------------------------------------------------------------------------

COLUMN_ALIGN = 256  # a rank's columns are whole tensor-core tiles (256 columns)


def column_ranges(n: int, world: int, align: int = COLUMN_ALIGN) -> List[Tuple[int, int]]:
    """Contiguous column ranges [c0, c1) of the ranks over the padded width
    n_pad (n rounded up to 128): multiples of `align` except the last end,
    as equal as whole `align` blocks allow (a rank may get none)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    n_pad = (int(n) + 127) // 128 * 128
    blocks = (n_pad + align - 1) // align
    out, b0 = [], 0
    for r in range(world):
        nb = blocks // world + (1 if r < blocks % world else 0)
        c0, c1 = min(b0 * align, n_pad), min((b0 + nb) * align, n_pad)
        out.append((c0, c1))
        b0 += nb
    return out


def assemble_columns(parts: Sequence, ranges: Sequence[Tuple[int, int]]):
    """Concatenate the ranks' column slices (arrays or tensors [B, n, words])
    along the last axis, in rank order: the full rows of n_pad / 64 words."""
    widths = [(c1 - c0) // 64 for c0, c1 in ranges]
    trimmed = [p[..., :w] for p, w in zip(parts, widths)]
    first = trimmed[0]
    if hasattr(first, "new_zeros"):  # torch
        import torch
        return torch.cat(list(trimmed), dim=-1)
    import numpy as np
    return np.concatenate(list(trimmed), axis=-1)


def all_gather_columns(local, ranges: Sequence[Tuple[int, int]], dist):
    """All-gather of every rank's column slice (a torch tensor [B, n, words]
    of int64 words; slices differ in width, so they travel padded to the
    widest) and their assembly into full rows."""
    import torch
    wmax = max((c1 - c0) // 64 for c0, c1 in ranges)
    pad = local.new_zeros(local.shape[:-1] + (wmax,))
    pad[..., : local.shape[-1]] = local
    parts = [torch.empty_like(pad) for _ in ranges]
    dist.all_gather(parts, pad)
    return assemble_columns(parts, ranges)


def run_column_sharded(engine, rank: int, world: int, dist=None, exchange=None) -> int:
    """Index creation of one query on this rank's columns, exchanging every
    iteration's new edges with the other ranks; returns the exchange steps
    (the iterations run; an engine may count one more that it can tell
    would add nothing).

    ``engine`` is this rank's closure: ``n``, ``begin(col0, col1)``,
    ``step()`` (one iteration of Listing 1 on the columns: the new edges of
    the iteration in those columns, [B, n, (col1 - col0) / 64] words) and
    ``apply(full)`` (the new edges of every column, [B, n, n_pad / 64]
    words, installed as the next iteration's A2; True once none was found).
    ``exchange(local, ranges)`` replaces the all-gather (default: over
    ``dist``, or the identity for one rank)."""
    ranges = column_ranges(engine.n, world)
    c0, c1 = ranges[rank]
    engine.begin(c0, c1)
    if exchange is None:
        if dist is not None and world > 1:
            exchange = lambda local, rg: all_gather_columns(local, rg, dist)  # noqa: E731
        else:
            exchange = lambda local, rg: local  # noqa: E731
    iters = 0
    while True:
        full = exchange(engine.step(), ranges)
        iters += 1
        if engine.apply(full):
            return iters


def run_column_sharded_lockstep(engines: Sequence) -> int:
    """The same protocol with every rank's engine in this process (ranks run
    one after another within an iteration; nothing waits on another rank's
    kernels): the all-gather is a concatenation.  Returns the steps."""
    world = len(engines)
    ranges = column_ranges(engines[0].n, world)
    for e, (c0, c1) in zip(engines, ranges):
        e.begin(c0, c1)
    iters = 0
    while True:
        parts = [e.step() for e in engines]
        full = assemble_columns(parts, ranges)
        iters += 1
        done = [e.apply(full) for e in engines]
        if all(done):
            return iters
        if any(done):
            raise RuntimeError("ranks disagree on the end of the loop")
