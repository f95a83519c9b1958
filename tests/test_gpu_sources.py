"""Multiple-source index creation (cfpq_run_sources): the rows of the
sources equal Oracle B's worklist solution from the same sources and the
full run's rows; a query whose transitions read a nonterminal is computed in
full."""
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


def _ctx(C, g, r, **kw):
    ctx = C.Context(**kw)
    ctx.load_graph(g)
    ctx.load_rsm(r)
    return ctx


@pytest.mark.parametrize("n,deg,seed,k", [(300, 2, 1, 1), (777, 3, 2, 10), (1500, 8, 3, 40), (2000, 2, 4, 200)])
def test_rpq_sources_equal_oracle(C, n, deg, seed, k):
    g, r = W.rpq_abc(n=n, out_deg=deg, seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed))
    src = sorted(set(rng.integers(0, n, k).tolist()))
    want = oracle.worklist(g, r, sources=src)[0]
    full = _ctx(C, g, r, no_single_cta=1)
    full.run()
    fb = full.reachable_bits(0)
    for mode in (C.CFPQ_CLOSURE_AUTO, C.CFPQ_CLOSURE_TC_FP8):
        ctx = _ctx(C, g, r, closure_mode=mode)
        st = ctx.run_sources(src)
        got = ctx.reachable_bits(0)
        assert (got[src] == want[src]).all()
        assert (got[src] == fb[src]).all()
        # unreached rows are empty, reached ones exact
        assert not (got & ~fb).any()
        assert st.iterations == 2 or got[src].sum() == 0


def test_sources_edge_cases(C):
    g, r = W.rpq_abc(n=400, out_deg=2, seed=9)
    ctx = _ctx(C, g, r)
    ctx.run_sources([])
    # no source: only the epsilon pairs (x, x) of the nullable start state
    got = ctx.reachable_bits(0)
    assert (got == np.eye(g.n, dtype=bool)).all() == bool(r.state_final[r.box_start[r.start_box]])
    assert not (got & ~np.eye(g.n, dtype=bool)).any()
    ctx.run_sources([5, 5, 5, 7])
    want = oracle.worklist(g, r, sources=[5, 7])[0]
    got = ctx.reachable_bits(0)
    assert (got[[5, 7]] == want[[5, 7]]).all()
    # all vertices: the full answer
    ctx.run_sources(list(range(g.n)))
    full = _ctx(C, g, r)
    full.run()
    assert (ctx.reachable_bits(0) == full.reachable_bits(0)).all()
    # a plain run afterwards computes every row again
    ctx.run()
    assert (ctx.reachable_bits(0) == full.reachable_bits(0)).all()
    with pytest.raises(C.CfpqError) as e:
        ctx.run_sources([g.n])
    assert e.value.status == C.CFPQ_ERR_INVALID_ARG


def test_sources_cfpq_computes_everything(C):
    g, r = W.dyck_zipf(512)
    ctx = _ctx(C, g, r)
    ctx.run_sources([0, 1, 2])
    full = _ctx(C, g, r)
    full.run()
    assert (ctx.reachable_bits(0) == full.reachable_bits(0)).all()


def test_paths_after_a_multiple_source_run(C):
    """After cfpq_run_sources only the sources' rows are exact: paths from a
    source equal Oracle C's, from another vertex the call is refused until a
    full run."""
    g, r = W.rpq_abc(n=24, out_deg=4, seed=3)
    ctx = _ctx(C, g, r)
    ctx.run_sources([3, 5])
    for vf in range(0, g.n, 3):
        got, _ = ctx.extract_paths(0, 3, vf, 6)
        assert got == oracle.brute_paths(g, r, 0, 3, vf, 6), vf
    with pytest.raises(C.CfpqError) as e:
        ctx.extract_paths(0, 4, 6, 6)
    assert e.value.status == C.CFPQ_ERR_INVALID_ARG
    ctx.run()
    got, _ = ctx.extract_paths(0, 4, 6, 6)
    assert got == oracle.brute_paths(g, r, 0, 4, 6, 6)
