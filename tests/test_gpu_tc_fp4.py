"""Index creation with the closure's products on block-scaled FP4 tensor-core
tiles (CFPQ_CLOSURE_TC_FP4, and AUTO's tiles in the FP4 format) is bit-exact
with the oracle and with the bit-packed closure.

The operands are 0/1 E2M1 values with every scale factor 1.0, so an output
element is the plain count of common ones (at most the inner dimension,
< 2^24, exact in FP32) and count > 0 is the Boolean product (Sec. 3.1's
closure).  The tiles are 256 x 192 output bits, so the sizes below include
n that are not multiples of 192 or 256 (ragged last tiles) and inner
dimensions that are not multiples of the 256-element K stage."""
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


def test_worked_example_fp4(C):
    g, r = W.worked_example()
    ctx, st, out = _run(g, r, C.CFPQ_CLOSURE_TC_FP4)
    assert out[0].tolist() == [[False, True], [False, True]]
    assert st.iterations == 3
    ref = oracle.kron_fixpoint(g, r, want_c=True)
    rows = [(s, x) for s in range(r.n_states) for x in range(g.n)]
    assert (ctx.closure_rows(rows) == ref.c).all()


@pytest.mark.parametrize("p,q", [(3, 4), (7, 8)])
def test_two_cycles_fp4(C, p, q):
    g, r = W.two_cycles(p, q)
    _, st, out = _run(g, r, C.CFPQ_CLOSURE_TC_FP4)
    assert st.iterations == p * q + 1
    assert (out == oracle.worklist(g, r)).all()


@pytest.mark.parametrize("n,deg,seed", [(48, 2, 1), (300, 3, 2), (1000, 8, 3)])
def test_rpq_fp4_equals_bitpacked_and_oracle(C, n, deg, seed):
    g, r = W.rpq_abc(n=n, out_deg=deg, seed=seed)
    c1, s1, a = _run(g, r, C.CFPQ_CLOSURE_TC_FP4)
    c2, s2, b = _run(g, r, C.CFPQ_CLOSURE_BITPACKED)
    assert (a == b).all() and (a == oracle.worklist(g, r)).all()
    assert s1.iterations == s2.iterations and s1.tile_mmas > 0
    rows = [(s, x) for s in range(r.n_states) for x in range(0, n, max(1, n // 13))]
    assert (c1.closure_rows(rows) == c2.closure_rows(rows)).all()


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("fmt", [2, 4])  # kind::mxf4 (UE8M0 scales), kind::mxf4nvf4 (UE4M3 scales)
def test_random_cfpq_fp4(C, seed, fmt):
    rng = np.random.Generator(np.random.PCG64(300 + seed))
    n = int(rng.integers(1, 500))
    g, r = W.small_random_instance(400 + seed, n=n, m=int(rng.integers(0, 4 * n + 1)),
                                   n_labels=int(rng.integers(1, 5)), max_states=16)
    _, s1, a = _run(g, r, C.CFPQ_CLOSURE_TC_FP4, tile_format=fmt)
    assert (a == oracle.worklist(g, r)).all()
    _, s2, b = _run(g, r, C.CFPQ_CLOSURE_TC_FP8)
    assert (a == b).all() and s1.iterations == s2.iterations


@pytest.mark.parametrize("n", [511, 1000, 2047])
def test_dyck_fp4_ragged(C, n):
    g, r = W.dyck_zipf(n, seed=11)
    _, s1, a = _run(g, r, C.CFPQ_CLOSURE_TC_FP4)
    assert s1.tile_mmas > 0
    assert (a == oracle.worklist(g, r)).all()


@pytest.mark.parametrize("n", [2048, 3001, 8192])
def test_auto_fp4_equals_fp8_and_bitpacked(C, n):
    """AUTO with FP4 tiles (the default format) and with FP8 tiles give the
    answer of the bit-packed closure; at n <= 3001 also Oracle B's."""
    g, r = W.dyck_zipf(n)
    _, s4, a = _run(g, r, C.CFPQ_CLOSURE_AUTO, no_single_cta=1, tile_format=C.CFPQ_TILES_FP4)
    _, s8, b = _run(g, r, C.CFPQ_CLOSURE_AUTO, no_single_cta=1, tile_format=C.CFPQ_TILES_FP8)
    _, sb, c = _run(g, r, C.CFPQ_CLOSURE_BITPACKED)
    assert s4.tile_mmas > 0 and s8.tile_mmas > 0
    assert (a == c).all() and (b == c).all()
    assert s4.iterations == sb.iterations == s8.iterations
    if n <= 3001:
        assert (a == oracle.worklist(g, r)).all()


def test_batch_fp4(C):
    qs = [W.dyck_zipf(n, seed=60 + i) for i, n in enumerate([300, 900, 2100])]
    qs += W.batched_queries(count=5, n_min=30, n_max=400, seed=18)
    for mode in (C.CFPQ_CLOSURE_TC_FP4, C.CFPQ_CLOSURE_AUTO):
        ctx = C.Context(closure_mode=mode)
        ctx.batch_run(qs)
        for i, (g, r) in enumerate(qs):
            want = oracle.worklist(g, r)
            for b in range(r.n_boxes):
                assert (ctx.batch_reachable_bits(i, b) == want[b]).all()
        ctx.close()


def test_tile_format_is_validated(C):
    with pytest.raises(C.CfpqError) as e:
        C.Context(tile_format=5)
    assert e.value.status == C.CFPQ_ERR_INVALID_ARG
