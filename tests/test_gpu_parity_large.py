"""Oracle parity at the sizes where the closure kernels change form.

* n = 8192, 16384, 32768 (rows of 8192-32768 bits): the column slices of the
  nonterminal adjacency, the cp.async ring of the general gather (rows of
  more than 8192 bits), the tile jobs' inner dimension capped at n/2 with the
  uncompacted tile kernel for longer lists.  The whole answer of every
  closure mode is compared with Oracle B's, stored as hashes by
  tests/golden/make_dyck_golden.py (Oracle B takes minutes to an hour at
  these sizes; the script calls only the oracle and the input generator).
* n = 65536, the Dyck-4 workload itself (Oracle B would take hours): at
  sampled rows x, the answer is a fixpoint of Listing 1's iteration.  The
  oracle rebuilds M3 from the GPU's M2, computes the closure row of the
  product vertex (q0, x) by search, and extracts it; the result must be the
  GPU's row x of M2 exactly.  Missing pairs derivable from present ones fail
  this, and so does a pair the closure cannot produce.
* The served workload (n = 32768, random grammars): every answer of a mix
  run on the server equals Oracle B's at sampled source rows.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_2103_14688_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "dyck4_zipf_oracle_b.json")


@pytest.fixture(scope="module")
def C():
    from paper_2103_14688_gb300 import cfpq
    cfpq.load()
    return cfpq


def _golden():
    return json.load(open(GOLDEN))


def _graph_sha256(g):
    h = hashlib.sha256()
    for a in (g.src, g.lbl, g.dst):
        h.update(np.ascontiguousarray(np.asarray(a, dtype="<u4")).tobytes())
    return h.hexdigest()


def _check_against_golden(words, case, block_rows):
    w = np.ascontiguousarray(words.astype("<u8"))
    if hashlib.sha256(w.tobytes()).hexdigest() == case["answer_sha256"]:
        return
    bad = [i * block_rows for i, want in enumerate(case["block_sha1"])
           if hashlib.sha1(w[i * block_rows:(i + 1) * block_rows].tobytes()).hexdigest() != want]
    raise AssertionError(f"answer differs from Oracle B in the {len(bad)} row blocks starting at {bad[:16]}")


SIZES = [8192, 16384, 32768]
MODES = [("auto", {}), ("bitpacked", {"closure_mode": 1}), ("tc_fp8", {"closure_mode": 2}),
         ("tc_fp4", {"closure_mode": 4}), ("auto_fp8_tiles", {"tile_format": 1}),
         ("auto_slices1", {"gather_slices": 1}), ("auto_slices3", {"gather_slices": 3})]


@pytest.mark.parametrize("n", SIZES)
def test_dyck_whole_answer_equals_oracle_b(C, n):
    gold = _golden()
    if str(n) not in gold["cases"]:
        pytest.skip(f"no stored Oracle B answer for n = {n}")
    case = gold["cases"][str(n)]
    g, r = W.dyck_zipf(n)
    assert _graph_sha256(g) == case["graph_sha256"], "the input generator drew a different graph"
    for name, kw in MODES:
        ctx = C.Context(**kw)
        ctx.load_graph(g)
        ctx.load_rsm(r)
        ctx.run()
        assert ctx.count_reachable(0) == case["pairs"], name
        _check_against_golden(ctx.reachable_words(0), case, gold["block_rows"])
        ctx.close()


def _fixpoint_rows(g, r, words, rows):
    """Oracle: row x of the answer re-derived from the given M2 (one more
    iteration of Listing 1 restricted to the product vertex (q0, x))."""
    q0 = int(r.box_start[r.start_box])
    crow = oracle.closure_rows_words(g, r, words.reshape(1, g.n, -1), [(q0, x) for x in rows])
    finals = [f for f in range(r.n_states) if r.state_final[f] and r.state_box[f] == r.start_box]
    out = []
    for k, x in enumerate(rows):
        row = np.zeros(g.n, dtype=bool)
        for f in finals:
            row |= crow[k, f * g.n:(f + 1) * g.n]
        if r.state_final[q0]:
            row[x] = True
        out.append(row)
    return out


def test_dyck_full_size_is_a_fixpoint_at_sampled_rows(C):
    g, r = W.dyck_zipf()
    assert g.n == 65536
    ctx = C.Context()
    ctx.load_graph(g)
    ctx.load_rsm(r)
    ctx.run()
    words = ctx.reachable_words(0)
    ctx.close()
    deg = np.bincount(np.asarray(g.src), minlength=g.n)
    rng = np.random.Generator(np.random.PCG64(65536))
    rows = sorted(set(rng.integers(0, g.n, 6).tolist()) | {int(np.argmax(deg))})
    for x, want in zip(rows, _fixpoint_rows(g, r, words, rows)):
        got = np.unpackbits(words[x].view(np.uint8), bitorder="little")[: g.n].astype(bool)
        assert (got == want).all(), (x, int(got.sum()), int(want.sum()))


def test_served_full_size_answers_equal_oracle_b_rows(C):
    wl = W.serving_workload(lam=300.0, n_queries=24, horizon_s=60.0)
    g = wl.graph
    srv = C.Server(g)
    ks = wl.choice.tolist()[:24]
    tickets = []
    for i, k in enumerate(ks):
        tickets.append((srv.submit(wl.pool[k]), k))
        if i % 4 == 3:
            srv.step()
    got = {}
    for _ in range(200000):
        srv.step()
        for t, k in tickets:
            if t not in got and srv.poll(t):
                r = wl.pool[k]
                got[t] = srv.result_words(t, r.start_box)
                srv.release(t)
        if len(got) == len(tickets):
            break
    assert len(got) == len(tickets)
    srv.close()
    rng = np.random.Generator(np.random.PCG64(32768))
    srcs = sorted(rng.choice(g.n, size=32, replace=False).tolist())
    for t, k in tickets:
        r = wl.pool[k]
        want = oracle.worklist_words(g, r, sources=srcs)[r.start_box]
        assert (got[t][srcs] == want[srcs]).all(), (t, k)
