"""Path extraction (Sec. 3.2, Listing 2) on graphs beyond the tiny cases:
the path sets equal Oracle C's (all paths up to a length whose word the box
accepts) on RPQ, Dyck and two-cycle graphs and on random grammars with
nullable nonterminals.  The device's backward layers prune the host's
enumeration; these cases check that the pruning loses no path."""
from collections import deque

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


def _ctx(C, g, r):
    ctx = C.Context()
    ctx.load_graph(g)
    ctx.load_rsm(r)
    ctx.run()
    return ctx


def _within(g, vs, L):
    """Vertices at most L edges from vs (labels ignored)."""
    adj = [[] for _ in range(g.n)]
    for s, d in zip(np.asarray(g.src).tolist(), np.asarray(g.dst).tolist()):
        adj[s].append(d)
    dist = {vs: 0}
    dq = deque([vs])
    while dq:
        v = dq.popleft()
        if dist[v] == L:
            continue
        for w in adj[v]:
            if w not in dist:
                dist[w] = dist[v] + 1
                dq.append(w)
    return sorted(dist)


def _pairs(g, ctx, box, L, rng, count):
    """(vs, vf) pairs: mostly vf reachable within L edges and in the answer,
    plus some that are not."""
    bits = ctx.reachable_bits(box)
    out = []
    for vs in rng.permutation(g.n)[: 4 * count].tolist():
        near = [v for v in _within(g, vs, L) if bits[vs, v]]
        if near:
            out.append((vs, int(rng.choice(near))))
        else:
            out.append((vs, int(rng.integers(0, g.n))))
        if len(out) == count:
            break
    return out


def _check(C, g, r, ctx, box, pairs, L):
    for vs, vf in pairs:
        got, trunc = ctx.extract_paths(box, vs, vf, L)
        want = oracle.brute_paths(g, r, box, vs, vf, L)
        assert got == want, (box, vs, vf, len(got), len(want))
        assert not trunc


@pytest.mark.parametrize("n,deg,seed,L", [(2048, 4, 1, 6), (8192, 8, 2, 4), (1000, 3, 3, 7)])
def test_rpq_paths_equal_oracle(C, n, deg, seed, L):
    g, r = W.rpq_abc(n=n, out_deg=deg, seed=seed)
    ctx = _ctx(C, g, r)
    rng = np.random.Generator(np.random.PCG64(seed))
    _check(C, g, r, ctx, 0, _pairs(g, ctx, 0, L, rng, 12), L)


@pytest.mark.parametrize("n,seed,L", [(400, 5, 8), (1500, 6, 6)])
def test_dyck_paths_equal_oracle(C, n, seed, L):
    g, r = W.dyck_zipf(n=n, k=4, seed=seed)
    ctx = _ctx(C, g, r)
    rng = np.random.Generator(np.random.PCG64(seed))
    _check(C, g, r, ctx, 0, _pairs(g, ctx, 0, L, rng, 10), L)


@pytest.mark.parametrize("p,q", [(3, 4), (5, 6)])
def test_two_cycles_paths_equal_oracle(C, p, q):
    """a^k b^k over two cycles: the paths that return to vertex 0 wind around
    the cycles; long bounds give nested nonterminal expansions."""
    g, r = W.two_cycles(p, q)
    ctx = _ctx(C, g, r)
    L = 2 * p * q + 2
    _check(C, g, r, ctx, 0, [(0, 0), (1, 0), (0, p)], L)


@pytest.mark.parametrize("seed", range(6))
def test_random_grammar_paths_equal_oracle(C, seed):
    """Random grammars with unit and empty rules, several boxes."""
    g, r = W.small_random_instance(900 + seed, n=12, m=30, n_labels=2, max_states=14)
    ctx = _ctx(C, g, r)
    rng = np.random.Generator(np.random.PCG64(900 + seed))
    L = 5
    for b in range(r.n_boxes):
        pairs = [(int(rng.integers(0, g.n)), int(rng.integers(0, g.n))) for _ in range(6)]
        pairs += _pairs(g, ctx, b, L, rng, 6)
        _check(C, g, r, ctx, b, pairs, L)


def test_paths_truncation_is_a_prefix(C):
    g, r = W.rpq_abc(n=24, out_deg=4, seed=3)
    ctx = _ctx(C, g, r)
    L = 6
    vs, vf = max(((a, b) for a in range(4) for b in range(g.n)),
                 key=lambda ab: len(oracle.brute_paths(g, r, 0, ab[0], ab[1], L)))
    full, trunc = ctx.extract_paths(0, vs, vf, L)
    assert not trunc and len(full) > 3
    assert full == oracle.brute_paths(g, r, 0, vs, vf, L)
    for k in (1, 2, 3):
        part, trunc = ctx.extract_paths(0, vs, vf, L, max_paths=k)
        assert part == full[:k] and trunc


def test_paths_cache_follows_the_result(C):
    """The enumerator's host copies and memo are kept between calls of one
    result: bounds in either order, and a new graph and run, give Oracle C's
    answers."""
    g1, r = W.rpq_abc(n=24, out_deg=4, seed=3)
    g2, _ = W.rpq_abc(n=24, out_deg=4, seed=4)
    ctx = _ctx(C, g1, r)
    for L in (6, 3, 7, 2):
        for vs, vf in ((3, 6), (0, 5), (7, 7)):
            got, _ = ctx.extract_paths(0, vs, vf, L)
            assert got == oracle.brute_paths(g1, r, 0, vs, vf, L), (L, vs, vf)
    ctx.load_graph(g2)
    ctx.run()
    for vs, vf in ((3, 6), (0, 5), (7, 7)):
        got, _ = ctx.extract_paths(0, vs, vf, 6)
        assert got == oracle.brute_paths(g2, r, 0, vs, vf, 6), (vs, vf)
