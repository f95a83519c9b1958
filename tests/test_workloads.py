"""The synthetic inputs follow their stated recipes (readings R13-R16 of the
design notes and the workload table): Zipf truncation for mean 3, the
two-cycle numbering, the RPQ graph's out-degree and labels, the Dyck RSM's
shape, and seeded determinism.  CPU only."""
import numpy as np

from paper_2103_14688_gb300 import workloads as W


def test_zipf_truncation_for_mean_three():
    k = W.zipf_kmax_for_mean(2.1, 3.0)
    assert k == 192

    def mean(kmax):
        x = np.arange(1, kmax + 1, dtype=np.float64)
        w = x ** -2.1
        return float((w * x).sum() / w.sum())

    assert mean(192) >= 3.0 > mean(191)


def test_zipf_graph_degrees():
    g = W.zipf_graph(65536, 8, seed=11)
    deg = np.bincount(np.asarray(g.src), minlength=g.n)
    assert deg.min() >= 1 and deg.max() <= 192
    assert abs(deg.mean() - 3.0) < 0.1
    assert set(np.unique(g.lbl).tolist()) <= set(range(8))


def test_two_cycles_numbering():
    g, r = W.two_cycles(63, 64)
    assert g.n == 126
    edges = set(zip(np.asarray(g.src).tolist(), np.asarray(g.lbl).tolist(), np.asarray(g.dst).tolist()))
    a = {(i, 0, (i + 1) % 63) for i in range(63)}
    b = {(0, 1, 63)} | {(63 + i, 1, 64 + i) for i in range(62)} | {(125, 1, 0)}
    assert edges == a | b


def test_rpq_graph_recipe():
    g, r = W.rpq_abc(n=8192, out_deg=8, seed=7)
    deg = np.bincount(np.asarray(g.src), minlength=g.n)
    assert (deg == 8).all()
    assert set(np.unique(g.lbl).tolist()) <= {0, 1, 2}
    assert r.n_states == 8 and r.n_trans == 14


def test_dyck_rsm_shape():
    r = W.dyck_rsm(4)
    assert r.n_states == 11 and r.n_boxes == 1
    assert int(np.asarray(r.state_final).sum()) == 1


def test_generators_are_seeded():
    g1, _ = W.dyck_zipf(n=1024, seed=5)
    g2, _ = W.dyck_zipf(n=1024, seed=5)
    assert (g1.src == g2.src).all() and (g1.dst == g2.dst).all() and (g1.lbl == g2.lbl).all()
