"""Metamorphic properties of the GPU path at sizes the oracle tests do not
reach: renaming vertices or RSM states permutes the answer (or leaves it
unchanged), and adding edges never removes a pair.  Every answer is also
compared with Oracle B, so a failure names the side that moved."""
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


def _answer(C, g, r, **kw):
    ctx = C.Context(**kw)
    ctx.load_graph(g)
    ctx.load_rsm(r)
    ctx.run()
    return np.stack([ctx.reachable_bits(b) for b in range(r.n_boxes)])


@pytest.mark.parametrize("seed", range(4))
def test_vertex_permutation(C, seed):
    g, r = W.small_random_instance(1300 + seed, n=700, m=2100, n_labels=3, max_states=14)
    perm = np.random.Generator(np.random.PCG64(seed)).permutation(g.n).astype(np.uint32)
    g2 = W.Graph(g.n, g.n_terminals, perm[g.src], g.lbl.copy(), perm[g.dst])
    a, b = _answer(C, g, r), _answer(C, g2, r)
    assert (a == oracle.worklist(g, r)).all()
    assert (b[:, perm][:, :, perm] == a).all()


@pytest.mark.parametrize("seed", range(4))
def test_state_renumbering(C, seed):
    g, r = W.small_random_instance(1400 + seed, n=600, m=1800, n_labels=2, max_states=16)
    perm = np.random.Generator(np.random.PCG64(seed)).permutation(r.n_states).astype(np.uint32)
    fin = np.zeros_like(r.state_final)
    fin[perm] = r.state_final
    sb = np.zeros_like(r.state_box)
    sb[perm] = r.state_box
    r2 = W.RSM(r.n_states, r.n_boxes, r.start_box, perm[r.box_start], sb, fin,
               perm[r.tr_from], r.tr_kind.copy(), r.tr_sym.copy(), perm[r.tr_to])
    a, b = _answer(C, g, r), _answer(C, g, r2)
    assert (a == oracle.worklist(g, r)).all()
    assert (a == b).all()


@pytest.mark.parametrize("seed", range(4))
def test_adding_edges_never_removes_answers(C, seed):
    g, r = W.small_random_instance(1500 + seed, n=800, m=1600, n_labels=2, max_states=14)
    rng = np.random.Generator(np.random.PCG64(seed))
    extra = 200
    g2 = W.Graph(g.n, g.n_terminals,
                 np.concatenate([g.src, rng.integers(0, g.n, extra).astype(np.uint32)]),
                 np.concatenate([g.lbl, rng.integers(0, g.n_terminals, extra).astype(np.uint32)]),
                 np.concatenate([g.dst, rng.integers(0, g.n, extra).astype(np.uint32)]))
    a, b = _answer(C, g, r), _answer(C, g2, r)
    assert (b == oracle.worklist(g2, r)).all()
    assert not (a & ~b).any()


def test_vertex_permutation_dense_tiles(C):
    """The same on Dyck-4 with n = 2048, where AUTO moves the dense S matrix's
    products to the tensor-core tiles."""
    g, r = W.dyck_zipf(2048)
    perm = np.random.Generator(np.random.PCG64(17)).permutation(g.n).astype(np.uint32)
    g2 = W.Graph(g.n, g.n_terminals, perm[g.src], g.lbl.copy(), perm[g.dst])
    answers = []
    for gg in (g, g2):
        ctx = C.Context(no_single_cta=1)
        ctx.load_graph(gg)
        ctx.load_rsm(r)
        st = ctx.run()
        assert st.tile_mmas > 0
        answers.append(ctx.reachable_bits(0))
    a, b = answers
    assert (a == oracle.worklist(g, r)[0]).all()
    assert (b[perm][:, perm] == a).all()
