"""Parity at the workloads' full sizes, in the launch configuration the
benchmark uses: sampled outputs the oracle can compute, or properties that hold
at any size."""
import numpy as np
import pytest

import oracle
from paper_2103_14688_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def C():
    from paper_2103_14688_gb300 import cfpq
    cfpq.load()
    return cfpq


def test_batched_512_queries(C):
    """Every query of the 512-query batch equals its solo run; the smallest
    ones also equal the oracle."""
    qs = W.batched_queries()
    assert len(qs) == 512
    ctx = C.Context()
    per, tot = ctx.batch_run(qs)
    solo = C.Context()
    order = sorted(range(len(qs)), key=lambda i: qs[i][0].n)
    for i, (g, r) in enumerate(qs):
        solo.load_graph(g)
        solo.load_rsm(r)
        st = solo.run()
        assert per[i].iterations == st.iterations
        for b in range(r.n_boxes):
            assert (ctx.batch_reachable_bits(i, b) == solo.reachable_bits(b)).all(), (i, b)
    for i in order[:12]:
        g, r = qs[i]
        want = oracle.worklist(g, r)
        for b in range(r.n_boxes):
            assert (ctx.batch_reachable_bits(i, b) == want[b]).all()


def test_served_full_graph_equals_solo(C):
    """Queries arriving while others run on the 32768-vertex resident graph
    give the same answer as alone."""
    wl = W.serving_workload(lam=300.0, n_queries=40, horizon_s=60.0)
    srv = C.Server(wl.graph)
    tickets = []
    for i, k in enumerate(wl.choice.tolist()):
        tickets.append((srv.submit(wl.pool[k]), k))
        if i % 4 == 3:
            srv.step()
    got = {}
    for _ in range(200000):
        srv.step()
        for t, k in tickets:
            if t not in got and srv.poll(t):
                got[t] = [srv.result_bits(t, b) for b in range(wl.pool[k].n_boxes)]
                srv.release(t)
        if len(got) == len(tickets):
            break
    assert len(got) == len(tickets)
    solo = C.Context()
    solo.load_graph(wl.graph)
    for t, k in tickets:
        solo.load_rsm(wl.pool[k])
        solo.run()
        for b in range(wl.pool[k].n_boxes):
            assert (got[t][b] == solo.reachable_bits(b)).all(), (t, k, b)


def _short_dyck_targets(g, x, max_len, k):
    """Vertices y reached from x by a walk of at most max_len edges whose
    word is a nonempty balanced word over k bracket pairs (labels o_i = i,
    c_i = k + i): a depth-first walk with an explicit bracket stack."""
    adj = [[] for _ in range(g.n)]
    for s, l, d in zip(g.src.tolist(), g.lbl.tolist(), g.dst.tolist()):
        adj[s].append((l, d))
    for v in range(g.n):
        adj[v] = sorted(set(adj[v]))
    out = set()
    stack = [(x, (), 0)]
    while stack:
        v, brackets, ln = stack.pop()
        if ln > 0 and not brackets:
            out.add(v)
        if ln == max_len or len(brackets) > max_len - ln:
            continue
        for l, d in adj[v]:
            if l < k:
                stack.append((d, brackets + (l,), ln + 1))
            elif brackets and brackets[-1] == l - k:
                stack.append((d, brackets[:-1], ln + 1))
    return out


def test_dyck_full_size_properties(C):
    """n = 65536: (1) every walk of at most 8 edges spelling a Dyck word joins
    a pair of the answer (S -> S S | o_i c_i | o_i S c_i derives exactly the
    nonempty balanced words); (2) renumbering the vertices renumbers the
    answer."""
    g, r = W.dyck_zipf()
    assert g.n == 65536
    ctx = C.Context()
    ctx.load_graph(g)
    ctx.load_rsm(r)
    ctx.run()
    ans = ctx.reachable_words(0)
    rng = np.random.Generator(np.random.PCG64(17))
    for x in rng.integers(0, g.n, 24).tolist():
        for y in _short_dyck_targets(g, x, 8, 4):
            assert (int(ans[x, y >> 6]) >> (y & 63)) & 1, (x, y)
    perm = rng.permutation(g.n).astype(np.uint32)
    g2 = W.Graph(g.n, g.n_terminals, perm[g.src], g.lbl.copy(), perm[g.dst])
    ctx2 = C.Context()
    ctx2.load_graph(g2)
    ctx2.load_rsm(r)
    ctx2.run()
    assert ctx2.count_reachable(0) == ctx.count_reachable(0)
    ans2 = ctx2.reachable_words(0)
    for x in rng.integers(0, g.n, 64).tolist():
        row = np.unpackbits(ans[x].view(np.uint8), bitorder="little")[: g.n].astype(bool)
        row2 = np.unpackbits(ans2[perm[x]].view(np.uint8), bitorder="little")[: g.n].astype(bool)
        assert (row2[perm] == row).all()


def test_dyck_sliced_gather_equals_unsliced(C):
    """n = 16384 (rows of 16384 bits): the row gather splits the nonterminal
    adjacency columns of a work item over several CTAs that merge with
    atomics; the answer equals the unsliced gather's and the tensor-core
    mode's, and the closure rows agree on a sample."""
    g, r = W.dyck_zipf(16384)
    outs = []
    for kw in ({"gather_slices": 1}, {}, {"gather_slices": 3}, {"closure_mode": C.CFPQ_CLOSURE_TC_FP8}):
        ctx = C.Context(**kw)
        ctx.load_graph(g)
        ctx.load_rsm(r)
        st = ctx.run()
        rows = [(s, x) for s in range(r.n_states) for x in range(0, g.n, 997)]
        outs.append((st.iterations, ctx.reachable_words(0), ctx.closure_rows(rows)))
        ctx.close()
    for it, words, crows in outs[1:]:
        assert it == outs[0][0]
        assert (words == outs[0][1]).all()
        assert (crows == outs[0][2]).all()
