"""The allocation-free staging entry point (cfpq_load_graph_device_noalloc).

It is for callers that cannot let the library allocate device memory while
they replace a graph, e.g. a service whose device memory is one pre-sized pool.
The test stages two graphs in a row through it, on a context whose adjacency
buffers were sized by one ordinary load, and checks that each query answer is
the one the ordinary cfpq_load_graph_device path gives.  It runs last and
stands alone: it builds every context it uses.
"""
import ctypes

import numpy as np
import pytest

from paper_2103_14688_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _dev(g):
    import torch
    d = torch.device("cuda", 0)
    return [torch.from_numpy(a.astype(np.int32)).to(d) for a in (g.src, g.lbl, g.dst)]


def _answer(ctx, r):
    return np.stack([ctx.reachable_bits(b) for b in range(r.n_boxes)])


def test_noalloc_staging_matches_ordinary_staging():
    from paper_2103_14688_gb300 import cfpq as C
    lib = C.load()
    n = 3000
    g0, r = W.rpq_abc(n=n, out_deg=4, seed=100)
    graphs = [W.rpq_abc(n=n, out_deg=4, seed=s)[0] for s in (101, 102)]

    na = C.Context()
    s0, l0, d0 = _dev(g0)
    na.load_graph_device(n, 3, s0, l0, d0)      # sizes the context's adjacency buffers
    na.load_rsm(r)
    for g in graphs:                            # two allocation-free calls in a row
        s, l, d = _dev(g)
        rc = lib.cfpq_load_graph_device_noalloc(na.h, n, 3, int(s.numel()), ctypes.c_void_p(s.data_ptr()),
                                                ctypes.c_void_p(l.data_ptr()), ctypes.c_void_p(d.data_ptr()))
        assert rc == C.CFPQ_OK, lib.cfpq_last_error(na.h)
        na.run()
        got = _answer(na, r)

        ref = C.Context()
        ref.load_graph_device(n, 3, s, l, d)
        ref.load_rsm(r)
        ref.run()
        assert (got == _answer(ref, r)).all()
        ref.close()


def test_noalloc_staging_rejects_what_it_cannot_hold():
    from paper_2103_14688_gb300 import cfpq as C
    lib = C.load()
    g, r = W.rpq_abc(n=256, out_deg=2, seed=7)
    s, l, d = _dev(g)
    ctx = C.Context()
    # no graph loaded yet: the context owns no adjacency buffers to write into
    rc = lib.cfpq_load_graph_device_noalloc(ctx.h, 256, 3, int(s.numel()), ctypes.c_void_p(s.data_ptr()),
                                            ctypes.c_void_p(l.data_ptr()), ctypes.c_void_p(d.data_ptr()))
    assert rc == C.CFPQ_ERR_BUFFER_TOO_SMALL
    ctx.load_graph_device(256, 3, s, l, d)
    # beyond the fixed workspace: n_terminals * n_vertices > 2^19
    rc = lib.cfpq_load_graph_device_noalloc(ctx.h, 65536, 16, int(s.numel()), ctypes.c_void_p(s.data_ptr()),
                                            ctypes.c_void_p(l.data_ptr()), ctypes.c_void_p(d.data_ptr()))
    assert rc == C.CFPQ_ERR_UNSUPPORTED


@pytest.mark.parametrize("mode", [1, 2])  # bit-packed rows; tensor-core tiles (0/1 FP8)
def test_noalloc_same_size_swap_context_free(mode):
    """A same-size swap under context-free queries.  The a^n b^n and Dyck-4
    RSMs read pure-terminal blocks (per-label bitmaps of rows with an edge)
    and, with tiles, the terminal bit rows: both come from the edges, so the
    run after an allocation-free swap must rebuild them for the new graph."""
    import oracle
    from paper_2103_14688_gb300 import cfpq as C
    lib = C.load()
    gs = sorted((W.dyck_zipf(2048, seed=s)[0] for s in (41, 42)), key=lambda g: -g.m)
    for r in (W.anbn_rsm(), W.dyck_rsm()):
        na = C.Context(closure_mode=mode, no_single_cta=1)
        s0, l0, d0 = _dev(gs[0])
        na.load_graph_device(gs[0].n, gs[0].n_terminals, s0, l0, d0)  # the larger edge list sizes the buffers
        na.load_rsm(r)
        na.run()
        for g in (gs[1], gs[0]):  # swap in the other graph, then the first one back
            s, l, d = _dev(g)
            rc = lib.cfpq_load_graph_device_noalloc(na.h, g.n, g.n_terminals, int(s.numel()),
                                                    ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(l.data_ptr()),
                                                    ctypes.c_void_p(d.data_ptr()))
            assert rc == C.CFPQ_OK, lib.cfpq_last_error(na.h)
            na.run()
            got = _answer(na, r)
            ref = C.Context(closure_mode=mode, no_single_cta=1)
            ref.load_graph(g)
            ref.load_rsm(r)
            ref.run()
            assert (got == _answer(ref, r)).all()
            ref.close()
            assert (got == oracle.worklist(g, r)).all()
        na.close()
