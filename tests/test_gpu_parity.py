"""Parity of the CUDA path (through the C ABI) with the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_2103_14688_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfpq():
    from paper_2103_14688_gb300 import cfpq as C
    C.load()
    return C


def _run(C, g, r, **opt):
    ctx = C.Context(**opt)
    ctx.load_graph(g)
    ctx.load_rsm(r)
    st = ctx.run()
    out = np.stack([ctx.reachable_bits(b) for b in range(r.n_boxes)])
    return ctx, st, out


def _two_cycle_answer(p, q):
    n = p + q - 1
    out = np.zeros((n, n), dtype=bool)
    bv = [0] + list(range(p, n))
    for x in range(p):
        out[x, bv] = True
    return out


def test_worked_example(cfpq):
    g, r = W.worked_example()
    ctx, st, out = _run(cfpq, g, r)
    want = np.zeros((2, 2), dtype=bool)
    want[0, 1] = want[1, 1] = True
    assert (out[0] == want).all()
    assert st.iterations == 3 and st.edges_added == 2
    ref = oracle.kron_fixpoint(g, r, want_c=True)
    rows = [(s, x) for s in range(r.n_states) for x in range(g.n)]
    assert (ctx.closure_rows(rows) == ref.c).all()
    pairs = ctx.reachable_pairs(0)
    assert pairs.tolist() == [[0, 1], [1, 1]]


@pytest.mark.parametrize("p,q", [(3, 4), (5, 6), (7, 8), (4, 9), (63, 64)])
@pytest.mark.parametrize("loop", [0, 1])
def test_two_cycles_closed_form(cfpq, p, q, loop):
    g, r = W.two_cycles(p, q)
    ctx, st, out = _run(cfpq, g, r, loop_mode=loop)
    assert (out[0] == _two_cycle_answer(p, q)).all()
    assert st.iterations == p * q + 1
    assert st.edges_added == p * q


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("n,deg", [(48, 2), (200, 3), (777, 8)])
def test_rpq_small_vs_oracle(cfpq, seed, n, deg):
    g, r = W.rpq_abc(n=n, out_deg=deg, seed=seed)
    ctx, st, out = _run(cfpq, g, r)
    ref = oracle.worklist(g, r)
    assert (out == ref).all()
    assert st.iterations <= 2
    rows = [(s, x) for s in range(r.n_states) for x in range(0, n, max(1, n // 17))]
    assert (ctx.closure_rows(rows) == oracle.closure_rows(g, r, out, rows)).all()


@pytest.mark.parametrize("seed", [4, 5])
def test_rpq_iteration_count_equals_oracle_a(cfpq, seed):
    """The multi-kernel loop counts the last iteration (the one that adds no
    edge) exactly as Listing 1 does, including when it skips running it
    because the new edges lie in boxes no transition reads."""
    C = cfpq
    g, r = W.rpq_abc(n=96, out_deg=3, seed=seed)
    ref = oracle.kron_fixpoint(g, r)
    for mode in (C.CFPQ_CLOSURE_AUTO, C.CFPQ_CLOSURE_TC_FP8):
        ctx = C.Context(closure_mode=mode, no_single_cta=1)
        ctx.load_graph(g)
        ctx.load_rsm(r)
        st = ctx.run()
        assert st.iterations == ref.iterations == 2
        assert (ctx.reachable_bits(0) == ref.m2[0]).all()


def test_rpq_full_size_whole_answer(cfpq):
    """The RPQ workload at its full size (n = 8192, 8 out-edges): the whole
    answer equals Oracle B's (about 20 s of one host core)."""
    g, r = W.rpq_abc()
    ctx, st, out = _run(cfpq, g, r)
    rng = np.random.Generator(np.random.PCG64(7))
    assert (ctx.reachable_words(0) == oracle.worklist_words(g, r)[0]).all()
    assert st.iterations == 2
    # closure rows of sampled product vertices = BFS over M3 (RPQ: M3 is fixed)
    rows = [(int(s), int(x)) for s, x in zip(rng.integers(0, r.n_states, 12), rng.integers(0, g.n, 12))]
    assert (ctx.closure_rows(rows) == oracle.closure_rows(g, r, out, rows)).all()


@pytest.mark.parametrize("seed", range(24))
def test_random_cfpq_vs_oracles(cfpq, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(rng.integers(1, 300))
    g, r = W.small_random_instance(seed, n=n, m=int(rng.integers(0, 4 * n + 1)), n_labels=int(rng.integers(1, 5)),
                                   max_states=16)
    ctx, st, out = _run(cfpq, g, r)
    assert (out == oracle.worklist(g, r)).all()
    if n <= 64:
        a = oracle.kron_fixpoint(g, r)
        assert st.iterations == a.iterations


@pytest.mark.parametrize("n", [256, 1024])
def test_dyck_vs_oracle(cfpq, n):
    g, r = W.dyck_zipf(n)
    ctx, st, out = _run(cfpq, g, r)
    assert (out == oracle.worklist(g, r)).all()


def test_nullable_and_unit_cycles(cfpq):
    gram = {0: [(), (("t", 0), ("n", 0), ("t", 1))]}
    r = W.grammar_to_rsm(gram, 1)
    g = W.make_graph(4, 2, [(0, 0, 1), (1, 1, 2), (2, 0, 3), (3, 1, 0)])
    _, st, out = _run(cfpq, g, r)
    assert (out == oracle.kron_fixpoint(g, r).m2).all()
    # S -> T | a, T -> S b | S : unit cycle between boxes
    gram = {0: [(("n", 1),), (("t", 0),)], 1: [(("n", 0), ("t", 1)), (("n", 0),)]}
    r = W.grammar_to_rsm(gram, 2)
    g = W.make_graph(5, 2, [(0, 0, 1), (1, 1, 2), (2, 1, 3), (3, 0, 4), (4, 1, 0)])
    _, st, out = _run(cfpq, g, r)
    assert (out == oracle.worklist(g, r)).all()


def test_edge_cases(cfpq):
    C = cfpq
    r = W.anbn_rsm()
    # no edges at all
    g = W.Graph(5, 2, np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    _, st, out = _run(C, g, r)
    assert not out.any() and st.iterations == 1
    # one vertex with self-loops
    g = W.make_graph(1, 2, [(0, 0, 0), (0, 1, 0)])
    _, st, out = _run(C, g, r)
    assert out[0, 0, 0]
    # labels the RSM does not read, duplicates
    g = W.make_graph(3, 4, [(0, 0, 1), (0, 0, 1), (1, 1, 2), (2, 3, 0), (0, 2, 2)])
    _, st, out = _run(C, g, r)
    assert (out == oracle.kron_fixpoint(g, r).m2).all()


def test_invalid_inputs(cfpq):
    C = cfpq
    ctx = C.Context()
    with pytest.raises(C.CfpqError) as e:
        ctx.run()
    assert e.value.status == C.CFPQ_ERR_STATE
    bad = W.Graph(3, 2, np.array([0], np.uint32), np.array([0], np.uint32), np.array([3], np.uint32))
    with pytest.raises(C.CfpqError) as e:
        ctx.load_graph(bad)
    assert e.value.status == C.CFPQ_ERR_INVALID_ARG
    r = W.anbn_rsm()
    bad_r = W.RSM(r.n_states, r.n_boxes, 0, r.box_start, r.state_box, r.state_final, r.tr_from, r.tr_kind,
                  np.array([0, 5, 1, 1], np.uint32), r.tr_to)
    with pytest.raises(C.CfpqError) as e:
        ctx.load_rsm(bad_r)
    assert e.value.status == C.CFPQ_ERR_INVALID_ARG
    # a terminal the graph does not have
    g = W.make_graph(2, 1, [(0, 0, 1)])
    ctx.load_graph(g)
    with pytest.raises(C.CfpqError) as e:
        ctx.load_rsm(r)
    assert e.value.status == C.CFPQ_ERR_INVALID_ARG


def test_iteration_cap_reports_timeout(cfpq):
    C = cfpq
    g, r = W.two_cycles(7, 8)
    ctx = C.Context(max_iterations=5)
    ctx.load_graph(g)
    ctx.load_rsm(r)
    with pytest.raises(C.CfpqError) as e:
        ctx.run()
    assert e.value.status == C.CFPQ_ERR_TIMEOUT
    # the partial index is readable and is a subset of the answer
    part = ctx.reachable_bits(0)
    assert part.sum() == 5 and not (part & ~_two_cycle_answer(7, 8)).any()


def test_repeat_runs_and_reload(cfpq):
    C = cfpq
    g, r = W.rpq_abc(n=500, out_deg=4, seed=9)
    ctx = C.Context()
    ctx.load_graph(g)
    ctx.load_rsm(r)
    ctx.run()
    a = ctx.reachable_bits(0)
    ctx.run()
    assert (ctx.reachable_bits(0) == a).all()
    g2, _ = W.rpq_abc(n=500, out_deg=4, seed=10)
    ctx.load_graph(g2)
    ctx.run()
    assert (ctx.reachable_bits(0) == oracle.worklist(g2, r)[0]).all()
    assert ctx.count_reachable(0) == int(oracle.worklist(g2, r)[0].sum())


def test_batch_matches_single_and_oracle(cfpq):
    C = cfpq
    qs = W.batched_queries(count=12, n_min=20, n_max=400, seed=5)
    ctx = C.Context()
    per, tot = ctx.batch_run(qs)
    for i, (g, r) in enumerate(qs):
        want = oracle.worklist(g, r)
        for b in range(r.n_boxes):
            assert (ctx.batch_reachable_bits(i, b) == want[b]).all(), (i, b)
        _, st, out = _run(C, g, r)
        assert per[i].iterations == st.iterations


def test_extract_paths_worked_example(cfpq):
    g, r = W.worked_example()
    ctx, _, _ = _run(cfpq, g, r)
    for vs, vf in [(1, 1), (0, 1), (0, 0)]:
        got, trunc = ctx.extract_paths(0, vs, vf, 8)
        assert got == oracle.brute_paths(g, r, 0, vs, vf, 8)
    got, trunc = ctx.extract_paths(0, 1, 1, 8, max_paths=1)
    assert got == [((1, 0, 0), (0, 0, 1), (1, 1, 1), (1, 1, 1))] and trunc


@pytest.mark.parametrize("seed", range(8))
def test_extract_paths_random(cfpq, seed):
    g, r = W.small_random_instance(40 + seed, n=5, m=9, n_labels=2, max_states=10)
    ctx, _, out = _run(cfpq, g, r)
    L = 6
    for b in range(r.n_boxes):
        for vs in range(g.n):
            for vf in range(g.n):
                got, _ = ctx.extract_paths(b, vs, vf, L)
                want = oracle.brute_paths(g, r, b, vs, vf, L)
                assert got == want, (b, vs, vf)
                for p in got:
                    assert oracle.rsm_accepts(r, g.n_terminals, b, [l for _, l, _ in p])


@pytest.mark.parametrize("seed", range(16))
def test_single_cta_path_equals_multi_kernel(cfpq, seed):
    """Small queries run their whole fixpoint in one CTA; the answer, the
    iteration count and the closure equal the multi-kernel loop's."""
    rng = np.random.Generator(np.random.PCG64(7000 + seed))
    n = int(rng.integers(1, 500))
    g, r = W.small_random_instance(7000 + seed, n=n, m=int(rng.integers(0, 3 * n + 1)),
                                   n_labels=int(rng.integers(1, 4)), max_states=12)
    c1, s1, a = _run(cfpq, g, r)
    c2, s2, b = _run(cfpq, g, r, no_single_cta=1)
    assert (a == b).all()
    assert s1.iterations == s2.iterations and s1.edges_added == s2.edges_added
    rows = [(s, x) for s in range(r.n_states) for x in range(0, n, max(1, n // 7))]
    assert (c1.closure_rows(rows) == c2.closure_rows(rows)).all()
    if n <= 200:
        assert (a == oracle.worklist(g, r)).all()


def test_single_cta_path_two_cycles_full(cfpq):
    g, r = W.two_cycles(63, 64)
    _, s1, a = _run(cfpq, g, r)
    _, s2, b = _run(cfpq, g, r, no_single_cta=1)
    assert s1.gpu_launches == 1 and s2.gpu_launches > 1
    assert (a == b).all() and s1.iterations == s2.iterations == 4033
