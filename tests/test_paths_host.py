"""Host side of path extraction (Sec. 3.2, Listing 2), on the CPU: the
library's enumerator (csrc/cfpq_paths_host.h), driven by
tests/paths_host_driver.cpp with the backward layers emulated from their
definition and M2 from Oracle B, returns exactly Oracle C's paths.  Several
queries run on one enumerator, so its memo, layer cache and growing length
bound are exercised as the library uses them."""
import ctypes
import hashlib
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_2103_14688_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2103_14688_gb300", "csrc")
SRC = os.path.join(HERE, "paths_host_driver.cpp")
HDR = os.path.join(CSRC, "cfpq_paths_host.h")


@pytest.fixture(scope="module")
def lib():
    h = hashlib.sha1(open(SRC, "rb").read() + open(HDR, "rb").read()).hexdigest()[:16]
    out = os.path.join(tempfile.gettempdir(), f"cfpq_paths_host_driver_{h}.so")
    if not os.path.exists(out):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I", CSRC, "-o", tmp, SRC])
        os.replace(tmp, out)
    return ctypes.CDLL(out)


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def _paths(lib, g, r, queries):
    """Paths of every (box, vs, vf, max_len) query, run in order on one
    enumerator."""
    tri = np.array(sorted(set(zip(np.asarray(g.src).tolist(), np.asarray(g.lbl).tolist(),
                                  np.asarray(g.dst).tolist()))), dtype=np.uint32).reshape(-1, 3)
    m2 = np.ascontiguousarray(oracle.worklist_words(g, r), dtype=np.uint64)
    u32 = lambda a: np.ascontiguousarray(np.asarray(a), dtype=np.uint32)
    bs, sb, tf, tk, ts, tt = (u32(x) for x in (r.box_start, r.state_box, r.tr_from, r.tr_kind, r.tr_sym, r.tr_to))
    fin = np.ascontiguousarray(np.asarray(r.state_final), dtype=np.uint8)
    q = u32(np.array(queries, dtype=np.uint32).reshape(-1))
    edge_cap, path_cap = 1 << 20, 1 << 16
    edges = np.zeros(3 * edge_cap, dtype=np.uint32)
    offs = np.zeros(path_cap + 1, dtype=np.uint64)
    per = np.zeros(len(queries), dtype=np.uint64)
    tri_c = np.ascontiguousarray(tri.reshape(-1)) if len(tri) else np.zeros(3, dtype=np.uint32)
    rc = lib.phd_paths(ctypes.c_uint32(g.n), ctypes.c_uint64(len(tri)), _p(tri_c), ctypes.c_uint32(r.n_states),
                       ctypes.c_uint32(r.n_boxes), _p(bs), _p(sb), _p(fin), ctypes.c_uint32(r.n_trans), _p(tf),
                       _p(tk), _p(ts), _p(tt), _p(m2), ctypes.c_uint32(len(queries)), _p(q), _p(edges),
                       ctypes.c_uint64(edge_cap), _p(offs), ctypes.c_uint64(path_cap), _p(per))
    assert rc == 0, rc
    out, k = [], 0
    for c in per.tolist():
        ps = []
        for i in range(k, k + int(c)):
            a, b = int(offs[i]), int(offs[i + 1])
            ps.append(tuple((int(edges[3 * j]), int(edges[3 * j + 1]), int(edges[3 * j + 2])) for j in range(a, b)))
        out.append(ps)
        k += int(c)
    return out


def _check(lib, g, r, queries):
    got = _paths(lib, g, r, queries)
    for (box, vs, vf, L), ps in zip(queries, got):
        assert ps == oracle.brute_paths(g, r, box, vs, vf, L), (box, vs, vf, L)


def test_worked_example(lib):
    g, r = W.worked_example()
    _check(lib, g, r, [(0, vs, vf, L) for L in (8, 3, 10) for vs in range(g.n) for vf in range(g.n)])


@pytest.mark.parametrize("seed", range(10))
def test_random_grammars(lib, seed):
    """Several boxes, unit and empty rules; bounds in both orders."""
    g, r = W.small_random_instance(300 + seed, n=7, m=14, n_labels=2, max_states=12)
    rng = np.random.Generator(np.random.PCG64(300 + seed))
    qs = []
    for L in (5, 2, 6):
        for _ in range(10):
            qs.append((int(rng.integers(0, r.n_boxes)), int(rng.integers(0, g.n)), int(rng.integers(0, g.n)), L))
    _check(lib, g, r, qs)


def test_two_cycles_nested(lib):
    """a^k b^k on cycles of 3 and 4: one path of 18 edges nests S nine deep."""
    g, r = W.two_cycles(3, 4)
    _check(lib, g, r, [(0, 0, 3, 26), (0, 1, 0, 26), (0, 0, 0, 26), (0, 2, 5, 20)])


def test_dyck_and_rpq(lib):
    g, r = W.dyck_zipf(n=120, k=2, seed=4)
    rng = np.random.Generator(np.random.PCG64(4))
    _check(lib, g, r, [(0, int(rng.integers(0, g.n)), int(rng.integers(0, g.n)), 6) for _ in range(12)])
    g, r = W.rpq_abc(n=40, out_deg=3, seed=5)
    _check(lib, g, r, [(0, vs, vf, 5) for vs in range(0, 40, 7) for vf in range(0, 40, 5)])


@pytest.mark.parametrize("seed", range(12))
def test_word_lengths_against_brute_force(lib, seed):
    """The lengths the enumerator lets a box spell are exactly those of the
    words (over two terminals, up to length 7) that the RSM accepts."""
    import itertools
    g, r = W.small_random_instance(700 + seed, n=4, m=6, n_labels=2, max_states=12)
    L = 7
    u32 = lambda a: np.ascontiguousarray(np.asarray(a), dtype=np.uint32)
    fin = np.ascontiguousarray(np.asarray(r.state_final), dtype=np.uint8)
    out = np.zeros(r.n_boxes * (L + 1), dtype=np.uint8)
    args = [u32(x) for x in (r.box_start, r.state_box)]
    tr = [u32(x) for x in (r.tr_from, r.tr_kind, r.tr_sym, r.tr_to)]
    rc = lib.phd_word_lengths(ctypes.c_uint32(r.n_states), ctypes.c_uint32(r.n_boxes), _p(args[0]), _p(args[1]),
                              _p(fin), ctypes.c_uint32(r.n_trans), _p(tr[0]), _p(tr[1]), _p(tr[2]), _p(tr[3]),
                              ctypes.c_uint32(L), _p(out))
    assert rc == 0
    got = out.reshape(r.n_boxes, L + 1).astype(bool)
    for b in range(r.n_boxes):
        for j in range(L + 1):
            want = any(oracle.rsm_accepts(r, g.n_terminals, b, list(w))
                       for w in itertools.product(range(g.n_terminals), repeat=j))
            assert got[b, j] == want, (b, j)


def test_small_distance_caches(lib, monkeypatch):
    """Distance caches that hold two entries (dropped as they fill) give the
    same paths."""
    monkeypatch.setenv("PHD_DIST_CACHE_ENTRIES", "2")
    g, r = W.dyck_zipf(n=24, k=2, seed=3)
    _check(lib, g, r, [(0, vs, vf, 6) for vs in range(g.n) for vf in range(g.n)])
    g, r = W.small_random_instance(305, n=7, m=14, n_labels=2, max_states=12)
    _check(lib, g, r, [(b, vs, vf, 5) for b in range(r.n_boxes) for vs in range(g.n) for vf in range(g.n)])
