"""Loading a second graph of the same size into one context (Theorem 1's
answer must follow the new edges).

Reloading keeps the plan and the work lists when the shape (n, n_terminals)
is unchanged, but everything the closure derived from the old edges -- the
per-label bitmaps of rows that have an edge, read by pure-terminal blocks
such as Dyck-4's C[y_i, F], and the terminal bit rows of the tensor-core
tiles -- must be rebuilt.  Each case loads two Zipf Dyck-4 graphs of the same
n one after the other and compares both answers with Oracle B.
"""
import numpy as np
import pytest

import oracle
from paper_2103_14688_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MODES = {"auto": 0, "bitpacked": 1, "tc_fp8": 2}


def _answer(ctx, r):
    return np.stack([ctx.reachable_bits(b) for b in range(r.n_boxes)])


def _dev(g):
    import torch
    d = torch.device("cuda", 0)
    return [torch.from_numpy(np.asarray(a).astype(np.int32)).to(d) for a in (g.src, g.lbl, g.dst)]


def _load(ctx, g, how):
    if how == "host":
        ctx.load_graph(g)
    else:
        s, l, d = _dev(g)
        ctx.load_graph_device(g.n, g.n_terminals, s, l, d)
        ctx._keep = (s, l, d)


@pytest.mark.parametrize("how", ["host", "device"])
@pytest.mark.parametrize("mode", ["auto", "bitpacked"])
def test_same_size_reload_dyck(how, mode):
    from paper_2103_14688_gb300 import cfpq as C
    graphs = [W.dyck_zipf(1024, seed=s) for s in (11, 12)]
    with C.Context(closure_mode=MODES[mode]) as ctx:
        ctx.load_rsm(graphs[0][1])
        for g, r in graphs:
            _load(ctx, g, how)
            ctx.run()
            assert (_answer(ctx, r) == oracle.worklist(g, r)).all()


@pytest.mark.parametrize("mode", ["auto", "tc_fp8"])
def test_same_size_reload_dyck_tensor_tiles(mode):
    """n = 2048: AUTO moves the dense S products to tiles; TC_FP8 also reads
    the terminal bit rows, rebuilt after the reload."""
    from paper_2103_14688_gb300 import cfpq as C
    graphs = [W.dyck_zipf(2048, seed=s) for s in (21, 22)]
    with C.Context(closure_mode=MODES[mode], no_single_cta=1) as ctx:
        ctx.load_rsm(graphs[0][1])
        for g, r in graphs:
            _load(ctx, g, "device")
            st = ctx.run()
            assert st.tile_mmas > 0
            assert (_answer(ctx, r) == oracle.worklist(g, r)).all()


def test_same_size_reload_then_rsm_change():
    """A reload followed by a new RSM (a^n b^n over the same labels): the
    new plan sees the new graph."""
    from paper_2103_14688_gb300 import cfpq as C
    g1, r1 = W.dyck_zipf(1024, seed=31)
    g2, _ = W.dyck_zipf(1024, seed=32)
    r2 = W.anbn_rsm()
    with C.Context() as ctx:
        ctx.load_graph(g1)
        ctx.load_rsm(r1)
        ctx.run()
        ctx.load_graph(g2)
        ctx.load_rsm(r2)
        ctx.run()
        assert (_answer(ctx, r2) == oracle.worklist(g2, r2)).all()
        ctx.load_rsm(r1)
        ctx.run()
        assert (_answer(ctx, r1) == oracle.worklist(g2, r1)).all()
