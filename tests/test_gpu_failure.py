"""Failure detection without a GPU fault: the kernels' spin-waits are bounded.
A wait on an mbarrier that nothing arrives at gives up after its limit and
reports it, and the context then computes a query correctly."""
import time

import pytest

import oracle
from paper_2103_14688_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    from paper_2103_14688_gb300 import cfpq
    cfpq.load()
    return cfpq


@pytest.mark.parametrize("limit_ns", [1000, 2_000_000, 200_000_000])
def test_bounded_wait_gives_up_and_the_context_stays_usable(C, limit_ns):
    ctx = C.Context()
    t0 = time.perf_counter()
    assert ctx.check_bounded_wait(limit_ns)
    elapsed = time.perf_counter() - t0
    assert elapsed < 5.0
    if limit_ns >= 200_000_000:
        assert elapsed >= 0.9 * limit_ns / 1e9  # it waited for the limit, not less
    g, r = W.worked_example()
    ctx.load_graph(g)
    ctx.load_rsm(r)
    ctx.run()
    assert (ctx.reachable_bits(0) == oracle.worklist(g, r)[0]).all()


def test_bounded_wait_rejects_unbounded_limits(C):
    ctx = C.Context()
    for bad in (0, 10_000_000_000):
        with pytest.raises(C.CfpqError) as e:
            ctx.check_bounded_wait(bad)
        assert e.value.status == C.CFPQ_ERR_INVALID_ARG
