"""Pins for the CPU oracle: values printed in the paper, closed forms, textbook
routines, brute force and invariants.  Nothing here touches the CUDA path."""
import collections
import itertools
import json
import os
import re

import numpy as np
import pytest

import oracle
from paper_2103_14688_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _pairs(mat, n):
    """Product-matrix bits as {((s, x), (t, y))}."""
    return {((int(a) // n, int(a) % n), (int(b) // n, int(b) % n)) for a, b in np.argwhere(mat)}


def _as_pairs(lst):
    return {(tuple(a), tuple(b)) for a, b in lst}


# --- Sec. 3.3 worked example -------------------------------------------------

def test_worked_example_trace_matches_paper():
    gold = json.load(open(os.path.join(GOLDEN, "worked_example.json")))
    g, r = W.worked_example()
    res = oracle.kron_fixpoint(g, r, max_iter=10, trace=True)
    n = g.n
    it = gold["iterations"]
    assert res.iterations == len(it) == 3
    # iteration 1: M3,(1) exactly as printed, closure = M3 + one length-2 path
    assert _pairs(res.trace_m3[0], n) == _as_pairs(it[0]["m3"])
    assert _pairs(res.trace_c[0], n) == _as_pairs(it[0]["closure_new"])
    # iterations 2 and 3: the M3 bits the text says are added
    for k in (1, 2):
        added = _pairs(res.trace_m3[k] & ~res.trace_m3[k - 1], n)
        assert added == _as_pairs(it[k]["m3_added"])
    # iteration 2: the three new closure paths named in the text are new
    new_c = _pairs(res.trace_c[1] & ~res.trace_c[0], n)
    assert _as_pairs(it[1]["closure_new_paths"]) <= new_c
    # one S edge per iteration, then none
    assert list(res.trace_new) == [len(x["new_edges_S"]) for x in it]
    assert {tuple(p) for p in np.argwhere(res.m2[0]).tolist()} == {tuple(p) for p in gold["result_S"]}


def test_worked_example_all_oracles_agree():
    g, r = W.worked_example()
    expect = np.zeros((1, 2, 2), dtype=bool)
    expect[0, 0, 1] = expect[0, 1, 1] = True
    assert (oracle.kron_fixpoint(g, r).m2 == expect).all()
    assert (oracle.worklist(g, r) == expect).all()
    assert (oracle.brute_reach(g, r, 8) == expect).all()


def test_worked_example_shortest_path():
    gold = json.load(open(os.path.join(GOLDEN, "worked_example.json")))
    g, r = W.worked_example()
    paths = oracle.brute_paths(g, r, 0, 1, 1, 6)
    names = {"a": 0, "b": 1}
    want = tuple((u, names[l], v) for u, l, v in gold["get_paths_1_1_S_shortest"])
    assert paths[0] == want
    # every returned path spells a^k b^k
    for p in paths:
        w = "".join("ab"[l] for _, l, _ in p)
        k = len(w) // 2
        assert w == "a" * k + "b" * k and k > 0


# --- two coprime cycles: closed form -----------------------------------------

def _two_cycle_answer(p, q):
    n = p + q - 1
    A = list(range(p))            # a-cycle vertices
    Bv = [0] + list(range(p, n))  # b-cycle vertices
    out = np.zeros((n, n), dtype=bool)
    for x in A:
        for y in Bv:
            out[x, y] = True
    return out


@pytest.mark.parametrize("p,q", [(3, 4), (5, 6), (7, 8), (4, 9)])
def test_two_cycles_closed_form_kron(p, q):
    """a^k b^k from x on the a-cycle must end the a-run at 0 (k = -x mod p), the
    b-run then ends at b-position k mod q; by the CRT every pair of the a-cycle
    and the b-cycle is reached and the largest minimal k is p*q, so the loop
    adds one edge per iteration for p*q iterations and stops on the next."""
    g, r = W.two_cycles(p, q)
    res = oracle.kron_fixpoint(g, r, max_iter=10000)
    assert (res.m2[0] == _two_cycle_answer(p, q)).all()
    assert res.iterations == p * q + 1
    assert list(res.trace_new) == [1] * (p * q) + [0]
    assert (oracle.worklist(g, r)[0] == _two_cycle_answer(p, q)).all()


def test_two_cycles_full_size():
    g, r = W.two_cycles(63, 64)
    assert g.n == 126
    want = _two_cycle_answer(63, 64)
    assert want.sum() == 4032
    assert (oracle.worklist(g, r)[0] == want).all()
    res = oracle.kron_fixpoint(g, r, max_iter=5000)
    assert res.iterations == 4033 and (res.m2[0] == want).all()


# --- regular queries -------------------------------------------------------------

def test_abc_dfa_is_the_regex():
    d = W.abc_dfa_rsm()
    for L in range(0, 9):
        for w in itertools.product(range(3), repeat=L):
            s = "".join("abc"[c] for c in w)
            assert oracle.rsm_accepts(d, 3, 0, list(w)) == bool(re.fullmatch(W.ABC_REGEX, s)), s


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_rpq_equals_product_automaton_bfs(seed):
    g, r = W.rpq_abc(n=48, out_deg=2, seed=seed)
    bfs = oracle.product_bfs(g, r, list(range(g.n)))
    a = oracle.kron_fixpoint(g, r, max_iter=10)
    b = oracle.worklist(g, r)
    assert (a.m2[0] == bfs).all()
    assert (b[0] == bfs).all()
    # RPQ: one appending iteration, then one that adds nothing
    assert a.iterations <= 2 and a.trace_new[-1] == 0
    # the empty word is in the language: the diagonal is answered
    assert bfs.diagonal().all()


def test_rpq_full_size_sampled_rows():
    g, r = W.rpq_abc()
    rows = list(range(0, g.n, 1024))
    b = oracle.worklist(g, r, sources=rows)
    bfs = oracle.product_bfs(g, r, rows)
    assert (b[0][rows] == bfs).all()


# --- context-free queries: two independent oracles and brute force -------------

@pytest.mark.parametrize("seed", range(12))
def test_kron_equals_worklist_random(seed):
    n = 6 + seed % 5 * 4
    g, r = W.small_random_instance(seed, n=n, m=3 * n, n_labels=2 + seed % 3)
    a = oracle.kron_fixpoint(g, r, max_iter=100000)
    b = oracle.worklist(g, r)
    assert (a.m2 == b).all()


@pytest.mark.parametrize("seed", range(10))
def test_brute_force_exact_on_dags(seed):
    """On a DAG every path has at most n-1 edges, so enumerating all paths up
    to n-1 edges gives the exact answer of the reachability semantics."""
    rng = np.random.Generator(np.random.PCG64(1000 + seed))
    n, m, L = 5, 8, 2 + seed % 2
    u = rng.integers(0, n, size=m)
    v = rng.integers(0, n, size=m)
    keep = u != v
    s, d = np.minimum(u, v)[keep], np.maximum(u, v)[keep]
    lbl = rng.integers(0, L, size=s.shape[0])
    g = W.Graph(n, L, s.astype(np.uint32), lbl.astype(np.uint32), d.astype(np.uint32))
    _, _, r = W.random_grammar(rng, L, 3, 10)
    a = oracle.kron_fixpoint(g, r)
    assert (a.m2 == oracle.brute_reach(g, r, n - 1)).all()
    assert (oracle.worklist(g, r) == a.m2).all()


def test_brute_reach_bound_is_exact():
    """On the chain 0 -a-> 1 ... -a-> k -b-> ... -b-> 2k with S -> a S b | a b
    the pair (k-i, k+i) needs exactly 2i edges, so brute_reach with bound L
    holds exactly the pairs with 2i <= L (an off-by-one in the bound fails)."""
    k = 4
    es = [(v, 0, v + 1) for v in range(k)] + [(v, 1, v + 1) for v in range(k, 2 * k)]
    g = W.make_graph(2 * k + 1, 2, es)
    r = W.grammar_to_rsm({0: [(("t", 0), ("n", 0), ("t", 1)), (("t", 0), ("t", 1))]}, 1)
    for L in range(0, 2 * k + 2):
        want = np.zeros((g.n, g.n), dtype=bool)
        for i in range(1, k + 1):
            if 2 * i <= L:
                want[k - i, k + i] = True
        assert (oracle.brute_reach(g, r, L)[0] == want).all(), L


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_subset_on_cyclic(seed):
    g, r = W.small_random_instance(500 + seed, n=4, m=6, n_labels=2)
    a = oracle.kron_fixpoint(g, r)
    br = oracle.brute_reach(g, r, 7)
    assert not (br & ~a.m2).any()


def test_nullable_grammar_epsilon_rule():
    """S -> a S b | eps: every vertex pairs with itself, and a b between
    distinct vertices joins them (needs the epsilon edges to take part in the
    product, not only to sit in M2)."""
    gram = {0: [(), (("t", 0), ("n", 0), ("t", 1))]}
    r = W.grammar_to_rsm(gram, 1)
    g = W.make_graph(4, 2, [(0, 0, 1), (1, 1, 2), (2, 0, 3), (3, 1, 0)])
    a = oracle.kron_fixpoint(g, r)
    want = np.eye(4, dtype=bool)
    want[0, 2] = want[2, 0] = True
    assert (a.m2[0] == want).all()
    assert (oracle.worklist(g, r)[0] == want).all()
    assert (oracle.brute_reach(g, r, 8)[0] == want).all()


# --- grammar -> RSM and the membership chart ----------------------------------

def _derivable(gram, nn, nt, k):
    """Words of length <= k over terminals derivable from each nonterminal:
    least fixpoint of L_N = union over alternatives of the concatenation of the
    symbols' sets, truncated at length k."""
    L = {a: set() for a in range(nn)}
    changed = True
    while changed:
        changed = False
        for a in range(nn):
            for alt in gram.get(a, []):
                acc = {()}
                for kind, sym in alt:
                    parts = {(sym,)} if kind == "t" else L[sym]
                    acc = {x + y for x in acc for y in parts if len(x) + len(y) <= k}
                    if not acc:
                        break
                new = acc - L[a]
                if new:
                    L[a] |= new
                    changed = True
    return L


@pytest.mark.parametrize("seed", range(8))
def test_grammar_rsm_language(seed):
    rng = np.random.Generator(np.random.PCG64(77 + seed))
    nt = 2
    gram, nn, r = W.random_grammar(rng, nt, 3, 14)
    k = 5
    L = _derivable(gram, nn, nt, k)
    for b in range(nn):
        acc = set()
        for ln in range(k + 1):
            for w in itertools.product(range(nt), repeat=ln):
                if oracle.rsm_accepts(r, nt, b, list(w)):
                    acc.add(w)
        assert acc == L[b], (gram, b)


def test_paper_box_for_anbn():
    """The CFG -> RSM construction gives the four-state box of Fig. 3."""
    gram = {0: [(("t", 0), ("n", 0), ("t", 1)), (("t", 0), ("t", 1))]}
    r = W.grammar_to_rsm(gram, 1)
    ref = W.anbn_rsm()
    assert r.n_states == 4
    got = set(zip(r.tr_from.tolist(), r.tr_kind.tolist(), r.tr_sym.tolist(), r.tr_to.tolist()))
    # states: 0 start, 1 final (shared), 2 after 'a', 3 after 'a S'
    relabel = {0: 0, 1: 3, 2: 1, 3: 2}
    got = {(relabel[a], k, s, relabel[b]) for a, k, s, b in got}
    want = set(zip(ref.tr_from.tolist(), ref.tr_kind.tolist(), ref.tr_sym.tolist(), ref.tr_to.tolist()))
    assert got == want


# --- closure invariants ---------------------------------------------------------

def _warshall(m):
    c = m.copy()
    for k in range(c.shape[0]):
        c |= np.outer(c[:, k], c[k, :])
    return c


@pytest.mark.parametrize("seed", range(4))
def test_closure_invariants(seed):
    g, r = W.small_random_instance(900 + seed, n=7, m=16, n_labels=2)
    a = oracle.kron_fixpoint(g, r, trace=True, want_c=True)
    m3 = a.trace_m3[-1]
    c = a.c
    assert not (m3 & ~c).any()                                   # C contains M3
    cc = (c.astype(np.uint8) @ c.astype(np.uint8)) > 0
    assert not (cc & ~c).any()                                   # C . C in C
    assert (c == _warshall(m3)).all()                            # = Warshall closure
    rows = [(s, x) for s in range(r.n_states) for x in range(g.n)]
    assert (oracle.closure_rows(g, r, a.m2, rows) == c).all()    # = BFS rows
    # the final C's start-to-final blocks are exactly M2 minus epsilon edges
    n = g.n
    for b in range(r.n_boxes):
        q0 = int(r.box_start[b])
        got = np.zeros((n, n), dtype=bool)
        for f in np.nonzero((r.state_box == b) & (r.state_final == 1))[0]:
            got |= c[q0 * n:(q0 + 1) * n, f * n:(f + 1) * n]
        if r.state_final[q0]:
            got |= np.eye(n, dtype=bool)
        assert (got == a.m2[b]).all()


@pytest.mark.parametrize("seed", range(3))
def test_monotone_growth(seed):
    g, r = W.small_random_instance(1200 + seed, n=8, m=20, n_labels=2)
    a = oracle.kron_fixpoint(g, r, trace=True)
    for k in range(1, a.iterations):
        assert not (a.trace_m3[k - 1] & ~a.trace_m3[k]).any()
        assert not (a.trace_c[k - 1] & ~a.trace_c[k]).any()


# --- metamorphic ------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
def test_vertex_permutation(seed):
    g, r = W.small_random_instance(300 + seed, n=12, m=30, n_labels=3)
    perm = np.random.Generator(np.random.PCG64(seed)).permutation(g.n).astype(np.uint32)
    g2 = W.Graph(g.n, g.n_terminals, perm[g.src], g.lbl.copy(), perm[g.dst])
    a = oracle.worklist(g, r)
    b = oracle.worklist(g2, r)
    assert (b[:, perm][:, :, perm] == a).all()


@pytest.mark.parametrize("seed", range(4))
def test_state_renumbering(seed):
    g, r = W.small_random_instance(400 + seed, n=10, m=24, n_labels=2)
    perm = np.random.Generator(np.random.PCG64(seed)).permutation(r.n_states).astype(np.uint32)
    fin = np.zeros_like(r.state_final)
    fin[perm] = r.state_final
    sb = np.zeros_like(r.state_box)
    sb[perm] = r.state_box
    r2 = W.RSM(r.n_states, r.n_boxes, r.start_box, perm[r.box_start], sb, fin,
               perm[r.tr_from], r.tr_kind.copy(), r.tr_sym.copy(), perm[r.tr_to])
    assert (oracle.kron_fixpoint(g, r2).m2 == oracle.kron_fixpoint(g, r).m2).all()


@pytest.mark.parametrize("seed", range(4))
def test_adding_edges_never_removes_answers(seed):
    g, r = W.small_random_instance(600 + seed, n=10, m=20, n_labels=2)
    rng = np.random.Generator(np.random.PCG64(seed))
    extra = 6
    g2 = W.Graph(g.n, g.n_terminals,
                 np.concatenate([g.src, rng.integers(0, g.n, extra).astype(np.uint32)]),
                 np.concatenate([g.lbl, rng.integers(0, g.n_terminals, extra).astype(np.uint32)]),
                 np.concatenate([g.dst, rng.integers(0, g.n, extra).astype(np.uint32)]))
    a, b = oracle.worklist(g, r), oracle.worklist(g2, r)
    assert not (a & ~b).any()


def test_duplicate_edges_are_merged():
    g, r = W.small_random_instance(31, n=9, m=20, n_labels=2)
    g2 = W.Graph(g.n, g.n_terminals, np.tile(g.src, 3), np.tile(g.lbl, 3), np.tile(g.dst, 3))
    assert (oracle.kron_fixpoint(g2, r).m2 == oracle.kron_fixpoint(g, r).m2).all()


def test_rejects_bad_input():
    g, r = W.worked_example()
    bad = W.Graph(2, 2, np.array([0], np.uint32), np.array([5], np.uint32), np.array([1], np.uint32))
    with pytest.raises(oracle.OracleError):
        oracle.kron_fixpoint(bad, r)
    bad = W.Graph(2, 2, np.array([0], np.uint32), np.array([0], np.uint32), np.array([2], np.uint32))
    with pytest.raises(oracle.OracleError):
        oracle.worklist(bad, r)


def _fixpoint_row(g, r, words, x):
    q0 = int(r.box_start[r.start_box])
    crow = oracle.closure_rows_words(g, r, words.reshape(1, g.n, -1), [(q0, x)])[0]
    row = np.zeros(g.n, dtype=bool)
    for f in range(r.n_states):
        if r.state_final[f] and r.state_box[f] == r.start_box:
            row |= crow[f * g.n:(f + 1) * g.n]
    return row


def test_fixpoint_row_check_accepts_the_answer_and_catches_dropped_pairs():
    """The full-size check of the GPU answer (one more iteration of Listing 1
    at a row, from a given M2) holds on Oracle B's answer and fails when
    pairs derivable from the rest are dropped (a mistake planted on the CPU),
    and closure_rows_words agrees with closure_rows."""
    g, r = W.dyck_zipf(512, seed=3)
    words = oracle.worklist_words(g, r)[0].copy()
    bits = oracle.worklist(g, r)
    rng = np.random.default_rng(0)
    xs = [int(x) for x in rng.integers(0, g.n, 12)]
    caught = 0
    for x in xs:
        row = np.unpackbits(words[x].view(np.uint8), bitorder="little")[: g.n].astype(bool)
        assert (_fixpoint_row(g, r, words, x) == row).all()
        ys = np.flatnonzero(row)
        if len(ys) < 4:
            continue
        # drop a quarter of the row's pairs; a dropped pair that another
        # derivation still yields from the remaining M2 shows up again
        drop = rng.choice(ys, size=len(ys) // 4, replace=False)
        bad = words.copy()
        for y in drop:
            bad[x, y >> 6] &= ~np.uint64(1 << (int(y) & 63))
        bad_row = np.unpackbits(bad[x].view(np.uint8), bitorder="little")[: g.n].astype(bool)
        caught += int((_fixpoint_row(g, r, bad, x) != bad_row).any())
    assert caught >= 1
    q0 = int(r.box_start[0])
    rows = [(q0, x) for x in xs[:3]] + [(1, xs[0])]
    assert (oracle.closure_rows_words(g, r, words.reshape(1, g.n, -1), rows) ==
            oracle.closure_rows(g, r, bits, rows)).all()


def test_fixpoint_check_of_every_box_on_generated_grammars():
    """The same check for every box of generated multi-box grammars (the
    batched workload's recipe, small n), including nullable boxes: each box
    b's row x is OR over finals f of b of C[(q0_b, x), (f, .)], plus (x, x)
    when q0_b is final.  Oracle B's answer passes at every row; one pair
    dropped from a row that keeps other pairs fails at that row for at least
    some rows of each query."""
    checked = 0
    cases = [W.small_random_instance(900 + seed, n=24, m=60, n_labels=3, max_states=14) for seed in range(6)]
    # S0 -> eps | a S1 b, S1 -> S0 c | c: a nullable box read by another
    gram = {0: [(), (("t", 0), ("n", 1), ("t", 1))], 1: [(("n", 0), ("t", 2)), (("t", 2),)]}
    rng = np.random.Generator(np.random.PCG64(906))
    es = [(int(rng.integers(0, 24)), int(rng.integers(0, 3)), int(rng.integers(0, 24))) for _ in range(70)]
    cases.append((W.make_graph(24, 3, es), W.grammar_to_rsm(gram, 2)))
    assert cases[-1][1].state_final[cases[-1][1].box_start[0]]
    for seed, (g, r) in enumerate(cases):
        words = oracle.worklist_words(g, r).copy()
        rows = [(int(r.box_start[b]), x) for b in range(r.n_boxes) for x in range(g.n)]
        crow = oracle.closure_rows_words(g, r, words, rows)

        def derived(b, x, c):
            q0 = int(r.box_start[b])
            row = np.zeros(g.n, dtype=bool)
            for f in range(r.n_states):
                if r.state_final[f] and r.state_box[f] == b:
                    row |= c[f * g.n:(f + 1) * g.n]
            if r.state_final[q0]:
                row[x] = True
            return row

        for k, (q0, x) in enumerate(rows):
            b = int(r.state_box[q0])
            have = np.unpackbits(words[b, x].view(np.uint8), bitorder="little")[: g.n].astype(bool)
            assert (derived(b, x, crow[k]) == have).all(), (seed, b, x)
        caught = 0
        for b in range(r.n_boxes):
            for x in range(g.n):
                ys = np.flatnonzero(np.unpackbits(words[b, x].view(np.uint8), bitorder="little")[: g.n])
                if len(ys) < 2:
                    continue
                bad = words.copy()
                bad[b, x, ys[0] >> 6] &= ~np.uint64(1 << (int(ys[0]) & 63))
                c = oracle.closure_rows_words(g, r, bad, [(int(r.box_start[b]), x)])[0]
                got = np.unpackbits(bad[b, x].view(np.uint8), bitorder="little")[: g.n].astype(bool)
                caught += int((derived(b, x, c) != got).any())
                checked += 1
        assert caught >= 1 or checked == 0, seed
    assert checked > 0


# --- all-path semantics (Oracle C), pinned by plain enumeration ------------------

def _walks(g, vs, vf, max_len):
    """Every walk vs -> vf of at most max_len edges, by depth-first search over
    the deduplicated edge set (a path is a sequence of (u, label, v) triples;
    paths may repeat vertices and edges)."""
    edges = sorted(set(zip(np.asarray(g.src).tolist(), np.asarray(g.lbl).tolist(), np.asarray(g.dst).tolist())))
    out = collections.defaultdict(list)
    for u, l, v in edges:
        out[u].append((u, l, v))
    found = []

    def dfs(x, path):
        if x == vf:
            found.append(tuple(path))
        if len(path) == max_len:
            return
        for e in out[x]:
            path.append(e)
            dfs(e[2], path)
            path.pop()

    dfs(vs, [])
    return found


@pytest.mark.parametrize("seed", range(6))
def test_brute_paths_complete_for_the_regex(seed):
    """Oracle C's paths of the RPQ (ab)*c|a*b* on small random graphs are
    exactly the walks whose word Python's re module accepts: a dropped or an
    extra path fails."""
    rng = np.random.Generator(np.random.PCG64(7000 + seed))
    n = int(rng.integers(2, 5))
    es = [(int(rng.integers(0, n)), int(rng.integers(0, 3)), int(rng.integers(0, n))) for _ in range(int(rng.integers(3, 8)))]
    g = W.make_graph(n, 3, es)
    r = W.abc_dfa_rsm()
    L = 5
    total = 0
    for vs in range(n):
        for vf in range(n):
            want = sorted((p for p in _walks(g, vs, vf, L)
                           if re.fullmatch(W.ABC_REGEX, "".join("abc"[l] for _, l, _ in p))),
                          key=lambda p: (len(p), p))
            assert oracle.brute_paths(g, r, 0, vs, vf, L) == want, (seed, vs, vf)
            total += len(want)
    assert total > 0


@pytest.mark.parametrize("seed", [0, 1, 2, 4, 5, 6])
def test_brute_paths_complete_for_anbn(seed):
    """The same for S -> a S b | a b (Fig. 3's box): the words a^k b^k, k >= 1,
    recognised by counting."""
    rng = np.random.Generator(np.random.PCG64(7100 + seed))
    n = int(rng.integers(2, 5))
    es = [(int(rng.integers(0, n)), int(rng.integers(0, 2)), int(rng.integers(0, n))) for _ in range(int(rng.integers(5, 10)))]
    g = W.make_graph(n, 2, es)
    r = W.anbn_rsm()

    def anbn(word):
        k = len(word) // 2
        return len(word) >= 2 and len(word) % 2 == 0 and word == [0] * k + [1] * k

    L = 6
    total = 0
    for vs in range(n):
        for vf in range(n):
            want = sorted((p for p in _walks(g, vs, vf, L) if anbn([l for _, l, _ in p])),
                          key=lambda p: (len(p), p))
            assert oracle.brute_paths(g, r, 0, vs, vf, L) == want, (seed, vs, vf)
            total += len(want)
    assert total > 0  # the seeds are chosen so that some pair has a path
