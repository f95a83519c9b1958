"""Multi-rank host logic on CPU: world_size 2 over gloo (no GPU)."""
import os
import socket

import pytest

from paper_2103_14688_gb300 import shard


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


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = [float(c) for c in range(1, 12)]
        # each query's "result" depends only on its index; ranks compute theirs
        res = shard.run_sharded(costs, rank, world, lambda idx: [i * i for i in idx], dist)
        mx = shard.max_over_ranks(10.0 + rank, dist)
        q.put((rank, res, mx))
    finally:
        dist.destroy_process_group()


def test_two_ranks_over_gloo():
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
    for rank, res, mx in out:
        assert res == [i * i for i in range(11)]
        assert mx == 11.0
