"""The tcgen05 Boolean-product tile kernel against a plain fp32 product."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ref(a, b):
    import torch
    return (torch.from_numpy(a.astype(np.float32)) @ torch.from_numpy(b.astype(np.float32)) > 0).numpy()


@pytest.mark.parametrize("n,p", [(1, 1.0), (7, 0.5), (128, 0.02), (200, 0.05), (256, 0.3), (300, 0.01),
                                 (513, 0.004), (1000, 0.002), (2048, 0.0005), (2048, 0.3)])
def test_tc_product_matches_fp32(n, p):
    from paper_2103_14688_gb300 import cfpq as C
    rng = np.random.Generator(np.random.PCG64(n * 1000 + int(p * 1000)))
    a = rng.random((n, n)) < p
    b = rng.random((n, n)) < p
    got = C.tc_bool_product(a, b)
    assert (got == _ref(a, b)).all()


def test_tc_product_structured():
    from paper_2103_14688_gb300 import cfpq as C
    n = 384
    eye = np.eye(n, dtype=bool)
    rng = np.random.Generator(np.random.PCG64(3))
    m = rng.random((n, n)) < 0.1
    assert (C.tc_bool_product(eye, m) == m).all()
    assert (C.tc_bool_product(m, eye) == m).all()
    z = np.zeros((n, n), dtype=bool)
    assert not C.tc_bool_product(z, m).any()
    full = np.ones((n, n), dtype=bool)
    assert C.tc_bool_product(full, full).all()   # counts of n = 384 are exact


def test_tc_int8_is_unsupported_on_sm103():
    from paper_2103_14688_gb300 import cfpq as C
    a = np.eye(4, dtype=bool)
    with pytest.raises(C.CfpqError) as e:
        C.tc_bool_product(a, a, use_int8=True)
    assert e.value.status == C.CFPQ_ERR_UNSUPPORTED
