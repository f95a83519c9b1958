"""Seeded synthetic inputs: labelled graphs, query automata and arrival streams.

This module is shared by the CUDA path, the oracle tests and the benchmark.  It
holds no step of the index-creation method (no Kronecker product, no closure, no
extraction): it only draws edge lists and writes down query automata.

Conventions (paper Sec. 2.1, Definition of an edge-labelled graph; Sec. 2.3,
Definition of an RSM):

* vertices are ``0..n-1``; an edge is a triple ``(src, label, dst)`` with
  ``label`` a terminal id ``0..n_terminals-1``; duplicates and self-loops may be
  present and are merged by every consumer (the graph is a set of edges);
* an RSM has ``n_states`` states numbered globally; box ``b`` owns the states
  with ``state_box[s] == b``, starts in ``box_start[b]`` and accepts in the
  states flagged by ``state_final``; a transition is ``(from, kind, sym, to)``
  with ``kind`` 0 for a terminal symbol and 1 for a call of box ``sym``.

Random numbers come from numpy's ``PCG64`` bit generator, seeded with
``SEED_BASE + config`` unless a seed is given.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

SEED_BASE = 2103_14688
TERM = 0
NONTERM = 1


@dataclasses.dataclass
class Graph:
    n: int
    n_terminals: int
    src: np.ndarray  # uint32 [m]
    lbl: np.ndarray  # uint32 [m]
    dst: np.ndarray  # uint32 [m]
    label_names: Optional[List[str]] = None

    @property
    def m(self) -> int:
        return int(self.src.shape[0])


@dataclasses.dataclass
class RSM:
    n_states: int
    n_boxes: int
    start_box: int
    box_start: np.ndarray    # uint32 [n_boxes]
    state_box: np.ndarray    # uint32 [n_states]
    state_final: np.ndarray  # uint8  [n_states]
    tr_from: np.ndarray      # uint32 [t]
    tr_kind: np.ndarray      # uint32 [t]
    tr_sym: np.ndarray       # uint32 [t]
    tr_to: np.ndarray        # uint32 [t]
    box_names: Optional[List[str]] = None

    @property
    def n_trans(self) -> int:
        return int(self.tr_from.shape[0])


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


def make_graph(n: int, n_terminals: int, edges: Sequence[Tuple[int, int, int]],
               label_names=None) -> Graph:
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 3)
    return Graph(n, n_terminals, _u32(e[:, 0]), _u32(e[:, 1]), _u32(e[:, 2]), label_names)


def make_rsm(n_states: int, box_start: Sequence[int], state_box: Sequence[int],
             finals: Sequence[int], transitions: Sequence[Tuple[int, int, int, int]],
             start_box: int = 0, box_names=None) -> RSM:
    fin = np.zeros(n_states, dtype=np.uint8)
    for f in finals:
        fin[f] = 1
    t = np.asarray(transitions, dtype=np.int64).reshape(-1, 4)
    return RSM(n_states, len(box_start), start_box, _u32(box_start), _u32(state_box),
               np.ascontiguousarray(fin), _u32(t[:, 0]), _u32(t[:, 1]), _u32(t[:, 2]),
               _u32(t[:, 3]), box_names)


# ---------------------------------------------------------------------------
# Grammars -> RSMs (one box per nonterminal, Sec. 2.3).
# ---------------------------------------------------------------------------
# A grammar is {nonterminal index: [alternative, ...]}, an alternative being a
# tuple of symbols ('t', id) or ('n', id).  Each box is the prefix trie of the
# alternatives of its nonterminal; the last symbol of every alternative enters
# one shared final state, the shape of the box drawn for S -> a S b | a b in
# Sec. 2.3 (four states, the prefix "a" shared, one final state).

Grammar = Dict[int, List[Tuple[Tuple[str, int], ...]]]


def grammar_to_rsm(grammar: Grammar, n_nonterminals: int, start: int = 0) -> RSM:
    box_start: List[int] = []
    state_box: List[int] = []
    finals: List[int] = []
    trans: List[Tuple[int, int, int, int]] = []
    for b in range(n_nonterminals):
        q0 = len(state_box)
        state_box.append(b)
        box_start.append(q0)
        final = len(state_box)
        state_box.append(b)
        finals.append(final)
        trie: Dict[Tuple, int] = {(): q0}
        edges = set()
        for alt in grammar.get(b, []):
            if len(alt) == 0:
                # epsilon alternative: the start state is also accepting
                finals.append(q0)
                continue
            cur = q0
            for i, (k, sym) in enumerate(alt):
                kind = TERM if k == 't' else NONTERM
                if i == len(alt) - 1:
                    nxt = final
                else:
                    key = tuple(alt[: i + 1])
                    if key not in trie:
                        trie[key] = len(state_box)
                        state_box.append(b)
                    nxt = trie[key]
                edges.add((cur, kind, sym, nxt))
                cur = nxt
        trans.extend(sorted(edges))
    return make_rsm(len(state_box), box_start, state_box, sorted(set(finals)), trans,
                    start_box=start)


# ---------------------------------------------------------------------------
# The worked example of Sec. 3.3: graph of Fig. 1, RSM of Fig. 3.
# ---------------------------------------------------------------------------

def worked_example() -> Tuple[Graph, RSM]:
    """Graph 0 -a-> 1, 1 -a-> 0, 1 -b-> 1 (Fig. 1) and the RSM of S -> a S b | a b
    with states 0..3, 0 -a-> 1, 1 -S-> 2, 1 -b-> 3, 2 -b-> 3, start 0, final 3
    (Fig. 3).  Terminals: a = 0, b = 1; box S = 0."""
    g = make_graph(2, 2, [(0, 0, 1), (1, 0, 0), (1, 1, 1)], ["a", "b"])
    r = make_rsm(4, [0], [0, 0, 0, 0], [3],
                 [(0, TERM, 0, 1), (1, NONTERM, 0, 2), (1, TERM, 1, 3), (2, TERM, 1, 3)],
                 box_names=["S"])
    return g, r


def anbn_rsm() -> RSM:
    """S -> a S b | a b as the four-state box of Fig. 3 (a = 0, b = 1)."""
    return worked_example()[1]


# ---------------------------------------------------------------------------
# Two coprime cycles sharing vertex 0 (S -> a S b | a b workload).
# ---------------------------------------------------------------------------

def two_cycles(p: int = 63, q: int = 64) -> Tuple[Graph, RSM]:
    """An a-labelled cycle 0 -> 1 -> ... -> p-1 -> 0 and a b-labelled cycle
    0 -> p -> p+1 -> ... -> p+q-2 -> 0 (q edges), n = p + q - 1 vertices.
    With p = 63, q = 64 this is the 126-vertex two-cycle graph."""
    n = p + q - 1
    edges = [(i, 0, (i + 1) % p) for i in range(p)]
    bcyc = [0] + list(range(p, p + q - 1))
    edges += [(bcyc[i], 1, bcyc[(i + 1) % q]) for i in range(q)]
    return make_graph(n, 2, edges, ["a", "b"]), anbn_rsm()


# ---------------------------------------------------------------------------
# Regular query (ab)*c | a*b* as a one-box RSM.
# ---------------------------------------------------------------------------

def abc_dfa_rsm() -> RSM:
    """Partial minimal DFA of (ab)*c | a*b* over a = 0, b = 1, c = 2.

    States are named by a shortest word reaching them:
    0 = eps, 1 = a, 2 = b, 3 = c, 4 = aa, 5 = ab, 6 = aba, 7 = abab;
    the dead state is left out.  Finals: eps, a, b, c, aa, ab."""
    a, b, c = 0, 1, 2
    tr = [
        (0, TERM, a, 1), (0, TERM, b, 2), (0, TERM, c, 3),
        (1, TERM, a, 4), (1, TERM, b, 5),
        (2, TERM, b, 2),
        (4, TERM, a, 4), (4, TERM, b, 2),
        (5, TERM, a, 6), (5, TERM, b, 2), (5, TERM, c, 3),
        (6, TERM, b, 7),
        (7, TERM, a, 6), (7, TERM, c, 3),
    ]
    return make_rsm(8, [0], [0] * 8, [0, 1, 2, 3, 4, 5], tr, box_names=["S"])


ABC_REGEX = r"(ab)*c|a*b*"


def random_out_degree_graph(n: int, out_deg: int, n_labels: int, seed: int) -> Graph:
    """Every vertex draws ``out_deg`` edges with uniform targets and uniform
    labels (duplicates are kept here and merged by the consumers)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    src = np.repeat(np.arange(n, dtype=np.uint32), out_deg)
    dst = rng.integers(0, n, size=n * out_deg, dtype=np.uint32)
    lbl = rng.integers(0, n_labels, size=n * out_deg, dtype=np.uint32)
    return Graph(n, n_labels, _u32(src), _u32(lbl), _u32(dst))


def rpq_abc(n: int = 8192, out_deg: int = 8, seed: Optional[int] = None) -> Tuple[Graph, RSM]:
    """Random graph with 8 uniform out-edges per vertex, labels uniform over
    {a, b, c}, queried with (ab)*c | a*b*."""
    seed = SEED_BASE + 2 if seed is None else seed
    g = random_out_degree_graph(n, out_deg, 3, seed)
    g.label_names = ["a", "b", "c"]
    return g, abc_dfa_rsm()


# ---------------------------------------------------------------------------
# Dyck-4 on a Zipf-degree graph.
# ---------------------------------------------------------------------------

def zipf_kmax_for_mean(alpha: float = 2.1, mean: float = 3.0, limit: int = 100000) -> int:
    """Smallest truncation point k_max of Zipf(alpha) on {1..k_max} whose mean
    is at least ``mean`` (2.1 and 3 give 192: the mean is 2.9997 at 191 and
    3.0017 at 192)."""
    k = np.arange(1, limit + 1, dtype=np.float64)
    w = k ** (-alpha)
    m = np.cumsum(w * k) / np.cumsum(w)
    idx = int(np.searchsorted(m, mean))
    return idx + 1


def zipf_graph(n: int, n_labels: int, seed: int, alpha: float = 2.1, mean: float = 3.0) -> Graph:
    """Out-degrees from Zipf(alpha) truncated to {1..k_max} (k_max chosen for the
    requested mean), uniform targets, uniform labels."""
    rng = np.random.Generator(np.random.PCG64(seed))
    kmax = zipf_kmax_for_mean(alpha, mean)
    k = np.arange(1, kmax + 1, dtype=np.float64)
    p = k ** (-alpha)
    p /= p.sum()
    deg = rng.choice(np.arange(1, kmax + 1), size=n, p=p).astype(np.int64)
    m = int(deg.sum())
    src = np.repeat(np.arange(n, dtype=np.uint32), deg)
    dst = rng.integers(0, n, size=m, dtype=np.uint32)
    lbl = rng.integers(0, n_labels, size=m, dtype=np.uint32)
    return Graph(n, n_labels, _u32(src), _u32(lbl), _u32(dst))


def dyck_rsm(k: int = 4) -> RSM:
    """S -> S S | o_i c_i | o_i S c_i (i = 1..k) as one box with 3 + 2k states:
    q0 = 0, p = 1, F = 2, x_i = 3 + i, y_i = 3 + k + i;
    q0 -S-> p -S-> F, q0 -o_i-> x_i -c_i-> F, x_i -S-> y_i -c_i-> F.
    Terminals: o_i = i, c_i = k + i (i = 0..k-1)."""
    q0, p, F = 0, 1, 2
    tr = [(q0, NONTERM, 0, p), (p, NONTERM, 0, F)]
    for i in range(k):
        x, y = 3 + i, 3 + k + i
        tr += [(q0, TERM, i, x), (x, TERM, k + i, F), (x, NONTERM, 0, y), (y, TERM, k + i, F)]
    n_states = 3 + 2 * k
    return make_rsm(n_states, [q0], [0] * n_states, [F], tr, box_names=["S"])


def dyck_zipf(n: int = 65536, k: int = 4, seed: Optional[int] = None) -> Tuple[Graph, RSM]:
    seed = SEED_BASE + 3 if seed is None else seed
    g = zipf_graph(n, 2 * k, seed)
    g.label_names = [f"o{i+1}" for i in range(k)] + [f"c{i+1}" for i in range(k)]
    return g, dyck_rsm(k)


# ---------------------------------------------------------------------------
# Seed-generated grammars (batched and served workloads).
# ---------------------------------------------------------------------------

def random_grammar(rng: np.random.Generator, n_terminals: int, min_states: int,
                   max_states: int, max_tries: int = 1000) -> Tuple[Grammar, int, RSM]:
    """1-4 nonterminals, 1-3 alternatives each, right-hand sides of length 1-3
    drawn uniformly over terminals and nonterminals; resampled until the RSM has
    between ``min_states`` and ``max_states`` states."""
    for _ in range(max_tries):
        nn = int(rng.integers(1, 5))
        gram: Grammar = {}
        for a in range(nn):
            alts = set()
            for _ in range(int(rng.integers(1, 4))):
                ln = int(rng.integers(1, 4))
                alt = []
                for _ in range(ln):
                    s = int(rng.integers(0, n_terminals + nn))
                    alt.append(('t', s) if s < n_terminals else ('n', s - n_terminals))
                alts.add(tuple(alt))
            gram[a] = sorted(alts)
        r = grammar_to_rsm(gram, nn)
        if min_states <= r.n_states <= max_states:
            return gram, nn, r
    raise RuntimeError("grammar generator did not reach the state range")


def er_graph(n: int, mean_out_deg: float, n_labels: int, rng: np.random.Generator) -> Graph:
    """G(n, m) with m = mean_out_deg * n uniform (src, dst) pairs, uniform labels."""
    m = int(round(mean_out_deg * n))
    src = rng.integers(0, n, size=m, dtype=np.uint32)
    dst = rng.integers(0, n, size=m, dtype=np.uint32)
    lbl = rng.integers(0, n_labels, size=m, dtype=np.uint32)
    return Graph(n, n_labels, _u32(src), _u32(lbl), _u32(dst))


def batched_queries(count: int = 512, n_min: int = 256, n_max: int = 8192,
                    seed: Optional[int] = None, min_states: int = 3,
                    max_states: int = 24) -> List[Tuple[Graph, RSM]]:
    """``count`` independent queries: n ~ U[n_min, n_max], Erdos-Renyi with mean
    out-degree 4 over 2-6 labels, RSM from :func:`random_grammar`."""
    seed = SEED_BASE + 4 if seed is None else seed
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        n = int(rng.integers(n_min, n_max + 1))
        nl = int(rng.integers(2, 7))
        g = er_graph(n, 4.0, nl, rng)
        _, _, r = random_grammar(rng, nl, min_states, max_states)
        out.append((g, r))
    return out


@dataclasses.dataclass
class ServingWorkload:
    graph: Graph
    pool: List[RSM]
    arrivals: np.ndarray   # float64 seconds, sorted
    choice: np.ndarray     # int64 index into pool


def serving_workload(n: int = 32768, pool_size: int = 256, lam: float = 100.0,
                     n_queries: int = 2000, horizon_s: float = 60.0,
                     seed: Optional[int] = None) -> ServingWorkload:
    """Resident Zipf graph (8 labels) and a pool of random RSMs with 3-32 states;
    Poisson arrivals at rate ``lam`` until ``n_queries`` or ``horizon_s``."""
    seed = SEED_BASE + 5 if seed is None else seed
    g = zipf_graph(n, 8, seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    pool = [random_grammar(rng, 8, 3, 32)[2] for _ in range(pool_size)]
    rng2 = np.random.Generator(np.random.PCG64(seed + 2 + int(lam * 1000)))
    gaps = rng2.exponential(1.0 / lam, size=n_queries)
    t = np.cumsum(gaps)
    t = t[t <= horizon_s]
    choice = rng2.integers(0, pool_size, size=t.shape[0])
    return ServingWorkload(g, pool, t, choice)


def small_random_instance(seed: int, n: int, m: int, n_labels: int,
                          min_states: int = 3, max_states: int = 12) -> Tuple[Graph, RSM]:
    """Tiny random CFPQ instance for oracle cross-checks."""
    rng = np.random.Generator(np.random.PCG64(seed))
    src = rng.integers(0, n, size=m, dtype=np.uint32)
    dst = rng.integers(0, n, size=m, dtype=np.uint32)
    lbl = rng.integers(0, n_labels, size=m, dtype=np.uint32)
    g = Graph(n, n_labels, _u32(src), _u32(lbl), _u32(dst))
    _, _, r = random_grammar(rng, n_labels, min_states, max_states)
    return g, r
