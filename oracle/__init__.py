"""Plain CPU oracle for Kronecker-product CFPQ/RPQ (arXiv 2103.14688).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  The C source
``cfpq_oracle.c`` shares nothing with the CUDA library; this module only
compiles it (gcc, once per source change) and marshals numpy arrays.

Results are numpy arrays of Booleans shaped ``[n_boxes, n, n]`` (reachability
per box, i.e. the final ``M2^N``) or ``[rows, Q*n]`` (closure rows, column index
``state * n + vertex`` as in Sec. 2.4).
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cfpq_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_lib = None


def build() -> str:
    """Compile the oracle into ``oracle/_build/`` and return the library path."""
    with open(_SRC, "rb") as f:
        digest = hashlib.sha1(f.read()).hexdigest()[:12]
    os.makedirs(_BUILD, exist_ok=True)
    so = os.path.join(_BUILD, f"libcfpq_oracle_{digest}.so")
    if not os.path.exists(so):
        tmp = so + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC]
        # OpenMP only spreads Oracle A's closure rows over threads when asked
        # (set_threads); without it the pragmas are ignored
        if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True).returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, so)
    return so


def set_threads(k: int) -> None:
    """Threads for the rows of Oracle A's closure (1 = sequential, the default)."""
    _load().orc_set_threads(ctypes.c_int(int(k)))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


def _wn(n: int) -> int:
    return (n + 63) // 64


def _unpack(words: np.ndarray, rows: int, bits: int) -> np.ndarray:
    w = words.reshape(rows, -1).view(np.uint8)
    return np.unpackbits(w, axis=1, bitorder="little")[:, :bits].astype(bool)


def _rsm_args(r):
    return [ctypes.c_uint32(r.n_states), ctypes.c_uint32(r.n_boxes), _p(_u32(r.box_start)),
            _p(_u32(r.state_box)), _p(np.ascontiguousarray(r.state_final, dtype=np.uint8)),
            ctypes.c_uint32(r.n_trans), _p(_u32(r.tr_from)), _p(_u32(r.tr_kind)),
            _p(_u32(r.tr_sym)), _p(_u32(r.tr_to))]


class _Keep:
    """Holds converted arrays alive for the duration of a C call."""

    def __init__(self, g, r):
        self.src, self.lbl, self.dst = _u32(g.src), _u32(g.lbl), _u32(g.dst)
        self.bs, self.sb = _u32(r.box_start), _u32(r.state_box)
        self.sf = np.ascontiguousarray(r.state_final, dtype=np.uint8)
        self.tf, self.tk, self.ts, self.tt = _u32(r.tr_from), _u32(r.tr_kind), _u32(r.tr_sym), _u32(r.tr_to)

    def graph(self, g):
        return [ctypes.c_uint32(g.n), ctypes.c_uint32(g.n_terminals), ctypes.c_uint64(len(self.src)),
                _p(self.src), _p(self.lbl), _p(self.dst)]

    def rsm(self, r, with_start_box=False):
        a = [ctypes.c_uint32(r.n_states), ctypes.c_uint32(r.n_boxes)]
        if with_start_box:
            a.append(ctypes.c_uint32(r.start_box))
        return a + [_p(self.bs), _p(self.sb), _p(self.sf), ctypes.c_uint32(r.n_trans),
                    _p(self.tf), _p(self.tk), _p(self.ts), _p(self.tt)]


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"{what} returned {rc}")


class KronResult:
    def __init__(self, m2, iters, trace_m3=None, trace_c=None, c=None, trace_new=None):
        self.m2 = m2                # bool [B, n, n]
        self.iterations = iters
        self.trace_m3 = trace_m3    # bool [iters, N, N] or None
        self.trace_c = trace_c
        self.c = c                  # bool [N, N] or None
        self.trace_new = trace_new  # int [iters] or None


def kron_fixpoint(g, r, max_iter: int = 100000, trace: bool = False,
                  want_c: bool = False) -> KronResult:
    """Oracle A (Listing 1, closure recomputed from scratch each iteration)."""
    lib = _load()
    k = _Keep(g, r)
    n, Q, B = g.n, r.n_states, r.n_boxes
    N = Q * n
    wn, wN = _wn(n), _wn(N)
    out_m2 = np.zeros(B * n * wn, dtype=np.uint64)
    iters = np.zeros(1, dtype=np.uint32)
    tm3 = np.zeros(max_iter * N * wN, dtype=np.uint64) if trace else None
    tc = np.zeros(max_iter * N * wN, dtype=np.uint64) if trace else None
    oc = np.zeros(N * wN, dtype=np.uint64) if want_c else None
    tnew = np.zeros(max_iter, dtype=np.uint64)
    rc = lib.orc_kron_fixpoint(*k.graph(g), *k.rsm(r), ctypes.c_uint32(max_iter), _p(out_m2), _p(iters),
                               _p(tm3) if trace else None, _p(tc) if trace else None,
                               _p(oc) if want_c else None, _p(tnew))
    _check(rc, "orc_kron_fixpoint")
    it = int(iters[0])
    m2 = _unpack(out_m2, B * n, n).reshape(B, n, n)
    res = KronResult(m2, it, trace_new=tnew[:it].astype(np.int64))
    if trace:
        res.trace_m3 = _unpack(tm3[: it * N * wN], it * N, N).reshape(it, N, N)
        res.trace_c = _unpack(tc[: it * N * wN], it * N, N).reshape(it, N, N)
    if want_c:
        res.c = _unpack(oc, N, N)
    return res


def worklist(g, r, sources: Optional[Sequence[int]] = None) -> np.ndarray:
    """Oracle B: Sum_b rows as bool [B, n, n] (rows of non-source vertices of
    the start box may be empty when ``sources`` is given)."""
    lib = _load()
    k = _Keep(g, r)
    n, B = g.n, r.n_boxes
    wn = _wn(n)
    out = np.zeros(B * n * wn, dtype=np.uint64)
    if sources is None:
        srcs, ns = None, 0
    else:
        srcs = _u32(sources)
        ns = len(srcs)
    rc = lib.orc_worklist(*k.graph(g), *k.rsm(r, with_start_box=True), ctypes.c_uint32(ns),
                          _p(srcs) if srcs is not None else None, _p(out))
    _check(rc, "orc_worklist")
    return _unpack(out, B * n, n).reshape(B, n, n)


def worklist_words(g, r, sources: Optional[Sequence[int]] = None) -> np.ndarray:
    """Oracle B with the raw bit rows, uint64 [B, n, ceil(n/64)]."""
    lib = _load()
    k = _Keep(g, r)
    n, B = g.n, r.n_boxes
    wn = _wn(n)
    out = np.zeros(B * n * wn, dtype=np.uint64)
    if sources is None:
        srcs, ns = None, 0
    else:
        srcs = _u32(sources)
        ns = len(srcs)
    rc = lib.orc_worklist(*k.graph(g), *k.rsm(r, with_start_box=True), ctypes.c_uint32(ns),
                          _p(srcs) if srcs is not None else None, _p(out))
    _check(rc, "orc_worklist")
    return out.reshape(B, n, wn)


def rsm_accepts(r, n_terminals: int, box: int, word: Sequence[int]) -> bool:
    lib = _load()
    w = _u32(list(word) if len(word) else [0])
    bs, sb = _u32(r.box_start), _u32(r.state_box)
    sf = np.ascontiguousarray(r.state_final, dtype=np.uint8)
    tf, tk, ts, tt = _u32(r.tr_from), _u32(r.tr_kind), _u32(r.tr_sym), _u32(r.tr_to)
    rc = lib.orc_rsm_accepts(ctypes.c_uint32(n_terminals), ctypes.c_uint32(r.n_states),
                             ctypes.c_uint32(r.n_boxes), _p(bs), _p(sb), _p(sf),
                             ctypes.c_uint32(r.n_trans), _p(tf), _p(tk), _p(ts), _p(tt),
                             ctypes.c_uint32(box), _p(w), ctypes.c_uint32(len(word)))
    if rc < 0:
        raise OracleError(f"orc_rsm_accepts returned {rc}")
    return bool(rc)


def brute_reach(g, r, max_len: int) -> np.ndarray:
    """Oracle C: pairs joined by a path of at most ``max_len`` edges whose word
    is accepted by box b, bool [B, n, n]."""
    lib = _load()
    k = _Keep(g, r)
    n, B = g.n, r.n_boxes
    out = np.zeros(B * n * _wn(n), dtype=np.uint64)
    rc = lib.orc_brute_reach(*k.graph(g), *k.rsm(r), ctypes.c_uint32(max_len), _p(out))
    _check(rc, "orc_brute_reach")
    return _unpack(out, B * n, n).reshape(B, n, n)


def brute_paths(g, r, box: int, vs: int, vf: int, max_len: int,
                path_cap: int = 1 << 16, edge_cap: int = 1 << 20) -> List[Tuple[Tuple[int, int, int], ...]]:
    """Oracle C for all-path semantics: every path vs -> vf with at most
    ``max_len`` edges whose word box ``box`` accepts, sorted by (length,
    triple sequence)."""
    lib = _load()
    k = _Keep(g, r)
    edges = np.zeros(edge_cap, dtype=np.uint32)
    off = np.zeros(path_cap + 1, dtype=np.uint64)
    npaths = np.zeros(1, dtype=np.uint64)
    rc = lib.orc_brute_paths(*k.graph(g), *k.rsm(r), ctypes.c_uint32(box), ctypes.c_uint32(vs),
                             ctypes.c_uint32(vf), ctypes.c_uint32(max_len), _p(edges),
                             ctypes.c_uint64(edge_cap), _p(off), ctypes.c_uint64(path_cap), _p(npaths))
    _check(rc, "orc_brute_paths")
    out = []
    for i in range(int(npaths[0])):
        a, b = int(off[i]), int(off[i + 1])
        out.append(tuple((int(edges[3 * j]), int(edges[3 * j + 1]), int(edges[3 * j + 2]))
                         for j in range(a, b)))
    out.sort(key=lambda p: (len(p), p))
    return out


def closure_rows(g, r, m2_nt: np.ndarray, rows: Sequence[Tuple[int, int]]) -> np.ndarray:
    """Rows of C = M3^+ for the nonterminal matrices ``m2_nt`` (bool [B, n, n]);
    result bool [len(rows), Q*n] indexed by state * n + vertex."""
    lib = _load()
    k = _Keep(g, r)
    n, Q, B = g.n, r.n_states, r.n_boxes
    N = Q * n
    wn, wN = _wn(n), _wn(N)
    m2 = np.asarray(m2_nt, dtype=bool).reshape(B * n, n)
    pad = np.zeros((B * n, wn * 64), dtype=bool)
    pad[:, :n] = m2
    words = np.packbits(pad, axis=1, bitorder="little").view(np.uint64).reshape(-1)
    words = np.ascontiguousarray(words)
    rs = _u32([a for a, _ in rows])
    rv = _u32([b for _, b in rows])
    out = np.zeros(len(rows) * wN, dtype=np.uint64)
    rc = lib.orc_closure_rows(*k.graph(g), *k.rsm(r), _p(words), ctypes.c_uint32(len(rows)), _p(rs), _p(rv),
                              _p(out))
    _check(rc, "orc_closure_rows")
    return _unpack(out, len(rows), N)


def closure_rows_words(g, r, m2_words: np.ndarray, rows: Sequence[Tuple[int, int]]) -> np.ndarray:
    """``closure_rows`` with the nonterminal matrices given as bit rows,
    uint64 [B, n, ceil(n/64)] (bit y of row x = word y/64, bit y%64): the
    form a large answer is read in.  Result bool [len(rows), Q*n]."""
    lib = _load()
    k = _Keep(g, r)
    n, Q, B = g.n, r.n_states, r.n_boxes
    N = Q * n
    wn, wN = _wn(n), _wn(N)
    words = np.ascontiguousarray(np.asarray(m2_words, dtype=np.uint64).reshape(B * n * wn))
    rs = _u32([a for a, _ in rows])
    rv = _u32([b for _, b in rows])
    out = np.zeros(len(rows) * wN, dtype=np.uint64)
    rc = lib.orc_closure_rows(*k.graph(g), *k.rsm(r), _p(words), ctypes.c_uint32(len(rows)), _p(rs), _p(rv),
                              _p(out))
    _check(rc, "orc_closure_rows")
    return _unpack(out, len(rows), N)


def product_bfs(g, dfa, sources: Sequence[int]) -> np.ndarray:
    """RPQ answer rows by breadth-first search over the product automaton
    graph x DFA (Sec. 2.4, Def. of FSM intersection): row i holds the vertices
    y reached from (start, sources[i]) in a final state, plus sources[i] itself
    when the start state is final (the empty word).  Plain Python; meant for
    a handful of sources."""
    n = g.n
    adj = [[[] for _ in range(n)] for _ in range(g.n_terminals)]
    for s, l, d in zip(g.src.tolist(), g.lbl.tolist(), g.dst.tolist()):
        adj[l][s].append(d)
    delta = [[] for _ in range(dfa.n_states)]
    for f, k, sym, t in zip(dfa.tr_from.tolist(), dfa.tr_kind.tolist(), dfa.tr_sym.tolist(),
                            dfa.tr_to.tolist()):
        if k != 0:
            raise OracleError("product_bfs needs a one-box RSM over terminals only")
        delta[f].append((sym, t))
    q0 = int(dfa.box_start[0])
    fin = dfa.state_final.astype(bool)
    out = np.zeros((len(sources), n), dtype=bool)
    for i, x in enumerate(sources):
        seen = np.zeros((dfa.n_states, n), dtype=bool)
        seen[q0, x] = True
        frontier = [(q0, x)]
        while frontier:
            nxt = []
            for s, v in frontier:
                for sym, t in delta[s]:
                    for w in adj[sym][v]:
                        if not seen[t, w]:
                            seen[t, w] = True
                            nxt.append((t, w))
            frontier = nxt
        out[i] = seen[fin].any(axis=0)
    return out
