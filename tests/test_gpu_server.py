"""Continuous-batching server: every answer equals its solo run and the oracle,
whatever the mix of queries running beside it."""
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


def _solo(C, g, r):
    ctx = C.Context()
    ctx.load_graph(g)
    ctx.load_rsm(r)
    ctx.run()
    return np.stack([ctx.reachable_bits(b) for b in range(r.n_boxes)])


def _drain(srv, tickets, max_steps=100000):
    for _ in range(max_steps):
        run, wait = srv.step()
        if all(srv.poll(t) for t in tickets) and run == 0 and wait == 0:
            return
    raise AssertionError("server did not finish")


def test_server_mix_equals_solo_and_oracle(C):
    wl = W.serving_workload(n=600, pool_size=24, lam=50.0, n_queries=40, seed=11)
    g = wl.graph
    srv = C.Server(g)
    tickets = []
    # queries arrive while others are running: submit in waves between steps
    order = list(wl.choice[:40])
    for i, k in enumerate(order):
        tickets.append((srv.submit(wl.pool[k]), k))
        if i % 3 == 2:
            srv.step()
    _drain(srv, [t for t, _ in tickets])
    for t, k in tickets:
        r = wl.pool[k]
        solo = _solo(C, g, r)
        for b in range(r.n_boxes):
            got = srv.result_bits(t, b)
            assert (got == solo[b]).all(), (t, k, b)
        srv.release(t)
    # spot-check a few against the oracle
    for k in sorted(set(order))[:6]:
        r = wl.pool[k]
        assert (_solo(C, g, r) == oracle.worklist(g, r)).all()


def test_server_admission_waits_for_memory(C):
    """A finished query keeps its device state until it is released; the
    client reads each result and releases it, which lets waiting queries in."""
    g, _ = W.dyck_zipf(1024, seed=3)
    rs = [W.dyck_rsm(), W.anbn_rsm(), W.dyck_rsm()]
    # budget that holds the graph and about one query at a time
    srv = C.Server(g, memory_budget=6 << 20)
    ts = [srv.submit(r) for r in rs]
    saw_waiting = False
    results = {}
    for _ in range(100000):
        run, wait = srv.step()
        saw_waiting |= wait > 0 and run > 0
        for t in ts:
            if t not in results and srv.poll(t):
                results[t] = srv.result_bits(t, 0)
                srv.release(t)
        if len(results) == len(ts):
            break
    assert saw_waiting and len(results) == len(ts)
    for t, r in zip(ts, rs):
        assert (results[t] == _solo(C, g, r)[0]).all()


def test_server_rejects_what_never_fits(C):
    g, r = W.dyck_zipf(2048, seed=4)
    srv = C.Server(g, memory_budget=8 << 20)
    t = srv.submit(r)
    with pytest.raises(C.CfpqError) as e:
        for _ in range(10):
            srv.step()
            srv.poll(t)
    assert e.value.status == C.CFPQ_ERR_OUT_OF_MEMORY


def test_server_release_of_waiting_query(C):
    g, r = W.dyck_zipf(512, seed=5)
    srv = C.Server(g)
    t1 = srv.submit(r)
    t2 = srv.submit(r)
    srv.release(t2)  # still waiting: cancelled
    _drain(srv, [t1])
    assert (srv.result_bits(t1, 0) == oracle.worklist(g, r)[0]).all()
    with pytest.raises(C.CfpqError):
        srv.poll(t2)


def test_server_cancel_running_query(C):
    """A running query released between steps is cancelled; the queries
    running beside it finish with their solo answers, and the server takes
    new work afterwards."""
    g, r = W.dyck_zipf(512, seed=6)
    qs = W.serving_workload(n=512, pool_size=6, seed=6)
    pool = [r] + list(qs.pool[:3])
    srv = C.Server(g)
    tickets = [srv.submit(x) for x in pool]
    run, _ = srv.step()
    assert run >= 1
    victim = tickets[0]
    assert not srv.poll(victim)  # still running: Dyck-4 needs many passes
    srv.release(victim)
    with pytest.raises(C.CfpqError):
        srv.poll(victim)
    rest = tickets[1:]
    _drain(srv, rest)
    for t, x in zip(rest, pool[1:]):
        want = _solo(C, g, x)
        for b in range(x.n_boxes):
            assert (srv.result_bits(t, b) == want[b]).all(), (t, b)
        srv.release(t)
    t2 = srv.submit(r)
    _drain(srv, [t2])
    assert (srv.result_bits(t2, 0) == oracle.worklist(g, r)[0]).all()
