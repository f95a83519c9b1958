"""Multi-rank host logic on CPU: world_size 2 over gloo (no GPU).

* Independent queries: ranks take a share of the batched workload
  (partition) and run it through the oracle; every rank ends with every
  query's answer.
* One query split by closure columns: every rank runs the column-restricted
  iteration of Listing 1 (here computed by the oracle's closure rows from the
  rank's M2, masked to its columns) and the ranks all-gather each
  iteration's new edges.  The answer and the iteration count must equal the
  unsharded oracles'.
"""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2103_14688_gb300 import shard
from paper_2103_14688_gb300 import workloads as W


def test_partition_is_complete_and_balanced():
    costs = [9, 1, 7, 3, 5, 5, 2, 8]
    parts = shard.partition(costs, 3)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(costs)))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(costs)
    assert shard.partition([], 2) == [[], []]
    assert shard.partition([1.0], 1) == [[0]]
    with pytest.raises(ValueError):
        shard.partition([1.0], 0)


def test_rank_seeds_differ():
    assert len({shard.rank_seed(100, r) for r in range(8)}) == 8


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _small_batch():
    return W.batched_queries(count=10, n_min=24, n_max=48, seed=5)


def _batch_answer(g, r):
    return oracle.worklist_words(g, r)


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        qs = _small_batch()
        costs = [shard.query_cost(g.n, r.n_states) for g, r in qs]
        res = shard.run_sharded(costs, rank, world, lambda idx: [_batch_answer(*qs[i]) for i in idx], dist)
        mx = shard.max_over_ranks(10.0 + rank, dist)
        q.put((rank, res, mx))
    finally:
        dist.destroy_process_group()


def test_two_ranks_over_gloo():
    """Each rank answers its share of a batch through the oracle; every rank
    ends with all answers."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = [_batch_answer(g, r) for g, r in _small_batch()]
    for rank, res, mx in out:
        assert len(res) == len(want)
        for a, b in zip(res, want):
            assert (a == b).all()
        assert mx == 11.0


class OracleColumnEngine:
    """A rank's closure for the column-sharded protocol, computed on the CPU
    by the oracle: one iteration of Listing 1 from the rank's M2 (the closure
    rows of every start-state product vertex, extracted), kept to the rank's
    columns.  M2 rows are n_pad / 64 words (n rounded up to 128)."""

    def __init__(self, g, r):
        self.g, self.r, self.n = g, r, g.n
        self.W = (g.n + 127) // 128 * 2
        self.m2 = None

    def begin(self, c0, c1):
        self.c0, self.c1 = c0, c1
        self.m2 = np.zeros((self.r.n_boxes, self.n, self.W), dtype=np.uint64)
        for b in range(self.r.n_boxes):  # the epsilon rows of Listing 1
            if self.r.state_final[self.r.box_start[b]]:
                for x in range(self.n):
                    self.m2[b, x, x >> 6] |= np.uint64(1 << (x & 63))

    def step(self):
        g, r, n = self.g, self.r, self.n
        wn = (n + 63) // 64
        rows = [(int(r.box_start[b]), x) for b in range(r.n_boxes) for x in range(n)]
        crow = oracle.closure_rows_words(g, r, self.m2[:, :, :wn], rows)
        new = np.zeros_like(self.m2)
        for b in range(r.n_boxes):
            fin = [f for f in range(r.n_states) if r.state_final[f] and r.state_box[f] == b]
            for x in range(n):
                row = np.zeros(self.W * 64, dtype=bool)
                for f in fin:
                    row[:n] |= crow[b * n + x, f * n:(f + 1) * n]
                row[: self.c0] = False
                row[self.c1:] = False
                new[b, x] = np.packbits(row, bitorder="little").view(np.uint64)
        new &= ~self.m2
        import torch
        return torch.from_numpy(new[:, :, self.c0 // 64:self.c1 // 64].view(np.int64).copy())

    def apply(self, full):
        full = np.asarray(full).view(np.uint64)
        self.m2 |= full
        return not full.any()


def _column_worker(rank, world, port, q, seed):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g, r = W.small_random_instance(seed, n=300, m=700, n_labels=3)
        e = OracleColumnEngine(g, r)
        iters = shard.run_column_sharded(e, rank, world, dist)
        q.put((rank, iters, e.m2))
    finally:
        dist.destroy_process_group()


def test_column_ranges_cover_the_padded_width():
    for n, world in ((300, 2), (300, 4), (1000, 3), (65536, 8), (129, 5)):
        rg = shard.column_ranges(n, world)
        n_pad = (n + 127) // 128 * 128
        assert rg[0][0] == 0 and rg[-1][1] == n_pad
        for (a0, a1), (b0, _) in zip(rg, rg[1:]):
            assert a1 == b0 and a0 <= a1
        assert all(c0 % 256 == 0 or c0 == c1 for c0, c1 in rg)


@pytest.mark.parametrize("seed", [1, 2])
def test_one_query_split_by_columns_over_gloo(seed):
    """Two ranks, one CFG query: the all-gathered answer equals Oracle B's and
    the loop runs as many iterations as Oracle A's unsharded loop."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_column_worker, args=(r, 2, port, q, seed)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g, r = W.small_random_instance(seed, n=300, m=700, n_labels=3)
    want = oracle.worklist_words(g, r)
    iters_a = oracle.kron_fixpoint(g, r).iterations
    wn = want.shape[-1]
    for rank, iters, m2 in out:
        assert (m2[:, :, :wn] == want).all()
        assert iters == iters_a


def test_one_query_split_by_columns_lockstep():
    """Four ranks in one process (the exchange is a concatenation), one of
    them without columns."""
    g, r = W.small_random_instance(3, n=300, m=700, n_labels=3)
    engines = [OracleColumnEngine(g, r) for _ in range(4)]
    iters = shard.run_column_sharded_lockstep(engines)
    want = oracle.worklist_words(g, r)
    wn = want.shape[-1]
    for e in engines:
        assert (e.m2[:, :, :wn] == want).all()
    assert iters == oracle.kron_fixpoint(g, r).iterations
