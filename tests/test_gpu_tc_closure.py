"""Index creation with the closure's products on the tensor cores
(CFPQ_CLOSURE_TC_FP8) is bit-exact with the oracle and with the bit-packed
closure."""
import numpy as np
import pytest

import oracle
from paper_2103_14688_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _run(g, r, mode, **kw):
    from paper_2103_14688_gb300 import cfpq as C
    ctx = C.Context(closure_mode=mode, **kw)
    ctx.load_graph(g)
    ctx.load_rsm(r)
    st = ctx.run()
    return ctx, st, np.stack([ctx.reachable_bits(b) for b in range(r.n_boxes)])


@pytest.fixture(scope="module")
def C():
    from paper_2103_14688_gb300 import cfpq
    cfpq.load()
    return cfpq


def test_worked_example_tc(C):
    g, r = W.worked_example()
    ctx, st, out = _run(g, r, C.CFPQ_CLOSURE_TC_FP8)
    assert out[0].tolist() == [[False, True], [False, True]]
    assert st.iterations == 3
    ref = oracle.kron_fixpoint(g, r, want_c=True)
    rows = [(s, x) for s in range(r.n_states) for x in range(g.n)]
    assert (ctx.closure_rows(rows) == ref.c).all()


@pytest.mark.parametrize("p,q", [(3, 4), (7, 8)])
def test_two_cycles_tc(C, p, q):
    g, r = W.two_cycles(p, q)
    _, st, out = _run(g, r, C.CFPQ_CLOSURE_TC_FP8)
    assert st.iterations == p * q + 1
    assert (out == oracle.worklist(g, r)).all()


@pytest.mark.parametrize("n,deg,seed", [(48, 2, 1), (300, 3, 2), (1000, 8, 3)])
def test_rpq_tc_equals_bitpacked_and_oracle(C, n, deg, seed):
    g, r = W.rpq_abc(n=n, out_deg=deg, seed=seed)
    c1, s1, a = _run(g, r, C.CFPQ_CLOSURE_TC_FP8)
    c2, s2, b = _run(g, r, C.CFPQ_CLOSURE_BITPACKED)
    assert (a == b).all() and (a == oracle.worklist(g, r)).all()
    assert s1.iterations == s2.iterations and s1.tile_mmas > 0
    rows = [(s, x) for s in range(r.n_states) for x in range(0, n, max(1, n // 13))]
    assert (c1.closure_rows(rows) == c2.closure_rows(rows)).all()


@pytest.mark.parametrize("seed", range(10))
def test_random_cfpq_tc(C, seed):
    rng = np.random.Generator(np.random.PCG64(100 + seed))
    n = int(rng.integers(1, 400))
    g, r = W.small_random_instance(200 + seed, n=n, m=int(rng.integers(0, 4 * n + 1)),
                                   n_labels=int(rng.integers(1, 5)), max_states=16)
    _, s1, a = _run(g, r, C.CFPQ_CLOSURE_TC_FP8)
    _, s2, b = _run(g, r, C.CFPQ_CLOSURE_BITPACKED)
    assert (a == b).all()
    assert (a == oracle.worklist(g, r)).all()
    assert s1.iterations == s2.iterations


@pytest.mark.parametrize("n", [512, 2048])
def test_dyck_tc(C, n):
    g, r = W.dyck_zipf(n)
    _, s1, a = _run(g, r, C.CFPQ_CLOSURE_TC_FP8)
    _, s2, b = _run(g, r, C.CFPQ_CLOSURE_BITPACKED)
    assert (a == b).all()
    assert (a == oracle.worklist(g, r)).all()


def test_batch_tc(C):
    qs = W.batched_queries(count=6, n_min=30, n_max=300, seed=8)
    ctx = C.Context(closure_mode=C.CFPQ_CLOSURE_TC_FP8)
    per, tot = ctx.batch_run(qs)
    for i, (g, r) in enumerate(qs):
        want = oracle.worklist(g, r)
        for b in range(r.n_boxes):
            assert (ctx.batch_reachable_bits(i, b) == want[b]).all()


def test_int8_mode_is_rejected(C):
    with pytest.raises(C.CfpqError) as e:
        C.Context(closure_mode=C.CFPQ_CLOSURE_TC_I8)
    assert e.value.status == C.CFPQ_ERR_UNSUPPORTED


@pytest.mark.parametrize("n", [512, 2048, 8192])
def test_auto_dense_tiles_dyck(C, n):
    """AUTO moves the products of Dyck-4's dense nonterminal matrix with the
    dirty closure rows to tensor-core tiles; the answer equals the row-gather
    closure and the oracle."""
    g, r = W.dyck_zipf(n)
    _, s1, a = _run(g, r, C.CFPQ_CLOSURE_AUTO, no_single_cta=1)
    _, s2, b = _run(g, r, C.CFPQ_CLOSURE_BITPACKED)
    assert (a == b).all()
    assert s1.iterations == s2.iterations
    if n >= 2048:                    # large enough to switch, and S is denser than 1/32: tiles ran
        assert s1.tile_mmas > 0 and s1.tile_kstages > 0
    if n <= 2048:
        assert (a == oracle.worklist(g, r)).all()


@pytest.mark.parametrize("seed", range(10))
def test_auto_random_dense_boxes(C, seed):
    rng = np.random.Generator(np.random.PCG64(900 + seed))
    n = int(rng.integers(20, 700))
    g, r = W.small_random_instance(900 + seed, n=n, m=int(rng.integers(n, 6 * n)),
                                   n_labels=int(rng.integers(1, 3)), max_states=14)
    c1, s1, a = _run(g, r, C.CFPQ_CLOSURE_AUTO, no_single_cta=1)
    c2, s2, b = _run(g, r, C.CFPQ_CLOSURE_BITPACKED, no_single_cta=1)
    assert (a == b).all() and s1.iterations == s2.iterations
    rows = [(s, x) for s in range(r.n_states) for x in range(0, n, max(1, n // 9))]
    assert (c1.closure_rows(rows) == c2.closure_rows(rows)).all()
    if n <= 300:
        assert (a == oracle.worklist(g, r)).all()


def test_auto_batch_dense_boxes(C):
    qs = [W.dyck_zipf(n, seed=40 + i) for i, n in enumerate([300, 700, 1200])]
    qs += W.batched_queries(count=5, n_min=100, n_max=600, seed=12)
    ctx = C.Context(closure_mode=C.CFPQ_CLOSURE_AUTO)
    per, tot = ctx.batch_run(qs)
    for i, (g, r) in enumerate(qs):
        want = oracle.worklist(g, r)
        for b in range(r.n_boxes):
            assert (ctx.batch_reachable_bits(i, b) == want[b]).all()
