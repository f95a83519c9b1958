"""One query split over ranks by closure columns, through the real closure
on the GPU.  The ranks run in one process on one GPU, one context each,
one after another within every iteration (no kernel waits on another
rank's); the all-gather of every iteration's new edges is a concatenation.
Every rank ends with the unsharded answer (and Oracle B's) after as many
iterations as the unsharded loop."""
import numpy as np
import pytest

import oracle
from paper_2103_14688_gb300 import shard
from paper_2103_14688_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    from paper_2103_14688_gb300 import cfpq
    cfpq.load()
    return cfpq


def _sharded(C, g, r, world, **opts):
    engines = [C.ColumnShardEngine(C.Context(no_single_cta=1, **opts), g, r) for _ in range(world)]
    iters = shard.run_column_sharded_lockstep(engines)
    answers = [np.stack([e.ctx.reachable_words(b) for b in range(r.n_boxes)]) for e in engines]
    stats = [e.stats() for e in engines]
    for e in engines:
        e.ctx.close()
    return iters, answers, stats


def _unsharded(C, g, r, **opts):
    with C.Context(**opts) as ctx:
        ctx.load_graph(g)
        ctx.load_rsm(r)
        st = ctx.run()
        return st, np.stack([ctx.reachable_words(b) for b in range(r.n_boxes)])


@pytest.mark.parametrize("world", [1, 2, 3])
@pytest.mark.parametrize("tile_format", [1, 2])
def test_dyck_split_by_columns(C, world, tile_format):
    """Dyck-4 at n = 2048: AUTO moves the dense S products (and, when they
    pay, the new-edge products) to tensor-core tiles, which every rank runs
    on its own columns (FP4 tiles are 192 columns wide, so some straddle a
    rank's 256-aligned column range and are masked)."""
    g, r = W.dyck_zipf(2048, seed=7)
    st, want = _unsharded(C, g, r, tile_format=tile_format)
    steps, answers, stats = _sharded(C, g, r, world, tile_format=tile_format)
    assert steps <= st.iterations
    for a, s in zip(answers, stats):
        assert (a == want).all()
        assert s.iterations == st.iterations
    assert (want[0] == oracle.worklist_words(g, r)[0]).all()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_grammars_split_by_columns(C, seed):
    g, r = W.small_random_instance(seed, n=700, m=2400, n_labels=3, max_states=16)
    want = oracle.worklist_words(g, r)
    for world, mode in ((2, 1), (4, 0)):
        steps, answers, stats = _sharded(C, g, r, world, closure_mode=mode)
        for a, s in zip(answers, stats):
            assert (a[:, :, :want.shape[-1]] == want).all()
            # Listing 1's iterations (an iteration that would only repeat
            # the last product is counted without running, as unsharded)
            assert s.iterations == oracle.kron_fixpoint(g, r).iterations
        assert steps <= stats[0].iterations


def test_rpq_split_by_columns_and_errors(C):
    g, r = W.rpq_abc(n=1500, out_deg=4, seed=3)
    st, want = _unsharded(C, g, r)
    steps, answers, stats = _sharded(C, g, r, 2)
    for a, s in zip(answers, stats):
        assert (a == want).all()
        assert s.iterations == st.iterations
    with C.Context() as ctx:
        ctx.load_graph(g)
        ctx.load_rsm(r)
        lib = ctx.lib
        assert lib.cfpq_shard_begin(ctx.h, 128, 256) == C.CFPQ_ERR_INVALID_ARG  # col0 not a multiple of 256
        assert lib.cfpq_shard_begin(ctx.h, 0, 4096) == C.CFPQ_ERR_INVALID_ARG   # beyond n_pad
        assert lib.cfpq_shard_step(ctx.h, None, None) == C.CFPQ_ERR_STATE      # no begin
