"""Checkpoint and resume (cfpq_set_start): the fixpoint of Listing 1 is
monotone, so a run started from pairs of the answer -- an earlier answer on
a subset of the edges, or the answer itself -- ends at the same answer
(Oracle B's), in no more iterations."""
import numpy as np
import pytest

import oracle
from paper_2103_14688_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    from paper_2103_14688_gb300 import cfpq
    cfpq.load()
    return cfpq


def _subgraph(g, keep, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    m = rng.random(len(g.src)) < keep
    return W.Graph(g.n, g.n_terminals, g.src[m].copy(), g.lbl[m].copy(), g.dst[m].copy())


def _words(ctx, B):
    return np.stack([ctx.reachable_words(b) for b in range(B)])


def _run(C, g, r, start=None, **kw):
    ctx = C.Context(**kw)
    ctx.load_graph(g)
    ctx.load_rsm(r)
    if start is not None:
        ctx.set_start(start)
    st = ctx.run()
    return ctx, st


@pytest.mark.parametrize("loop", ["device", "host"])
@pytest.mark.parametrize("seed", range(6))
def test_resume_from_a_subgraph_answer(C, seed, loop):
    lm = C.CFPQ_LOOP_DEVICE if loop == "device" else C.CFPQ_LOOP_HOST
    g, r = W.small_random_instance(2100 + seed, n=300, m=900, n_labels=2, max_states=14)
    sub = _subgraph(g, 0.7, seed)
    c0, _ = _run(C, sub, r, loop_mode=lm)
    start = _words(c0, r.n_boxes)
    c1, full = _run(C, g, r, loop_mode=lm)
    c2, resumed = _run(C, g, r, start=start, loop_mode=lm)
    want = oracle.worklist(g, r)
    for b in range(r.n_boxes):
        assert (c2.reachable_bits(b) == want[b]).all(), b
        assert (c1.reachable_bits(b) == want[b]).all(), b
    assert resumed.iterations <= full.iterations


def test_resume_from_the_answer_itself_dense_tiles(C):
    """Dyck-4 with n = 2048 (AUTO moves the dense S products to the tiles):
    started from its own answer, one iteration confirms the fixpoint."""
    g, r = W.dyck_zipf(2048)
    c1, full = _run(C, g, r, no_single_cta=1)
    ans = _words(c1, 1)
    c2, resumed = _run(C, g, r, start=ans, no_single_cta=1)
    assert (_words(c2, 1) == ans).all()
    assert (c2.reachable_bits(0) == oracle.worklist(g, r)[0]).all()
    assert full.iterations > 3 and resumed.iterations <= 2


def test_resume_rpq_from_half_the_edges(C):
    g, r = W.rpq_abc(n=4096, out_deg=6, seed=21)
    sub = _subgraph(g, 0.5, 21)
    c0, _ = _run(C, sub, r)
    c2, _ = _run(C, g, r, start=_words(c0, 1))
    c1, _ = _run(C, g, r)
    assert (_words(c2, 1) == _words(c1, 1)).all()


def test_worked_example_from_a_partial_answer(C):
    g, r = W.worked_example()
    start = np.zeros((1, g.n, 1), dtype=np.uint64)
    start[0, 0, 0] = 1 << 1  # (0, 1), the pair of the first iteration
    c, st = _run(C, g, r, start=start)
    assert (c.reachable_bits(0) == oracle.worklist(g, r)[0]).all()


def test_start_errors_and_clearing(C):
    g, r = W.worked_example()
    ctx = C.Context()
    ctx.load_graph(g)
    ctx.load_rsm(r)
    ctx.set_start(np.zeros((1, g.n + 1, 1), dtype=np.uint64))  # wrong vertex count
    with pytest.raises(C.CfpqError) as e:
        ctx.run()
    assert e.value.status == C.CFPQ_ERR_INVALID_ARG
    ctx.set_start(np.zeros((1, g.n, 1), dtype=np.uint64))
    with pytest.raises(C.CfpqError) as e:
        ctx.run_sources([0])
    assert e.value.status == C.CFPQ_ERR_STATE
    ctx.set_start(None)
    ctx.run()
    assert (ctx.reachable_bits(0) == oracle.worklist(g, r)[0]).all()
