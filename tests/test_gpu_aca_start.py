"""ACA start and restart rows: blocks whose rows far from the interface underflow
(squared-exponential, ell = 0.01 on [-1, 1]) keep their rank because the cross starts at
the row nearest the split; both forms match dense Cholesky and the oracle's ranks."""
import numpy as np
import pytest

import oracle as O
from paper_1403_6015_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_1403_6015_gb300 import build_lib, hodlr
    build_lib.build()
    hodlr.load()
    return hodlr


@pytest.mark.parametrize("precision", [0, 1])
def test_far_field_underflow(H, precision):
    n = 8192
    x, y = I.workload_1d(n, 1002)
    th, s2 = [0.01, 1.0], 1e-2
    h = H.Hodlr(x, "se", th, s2, 64, 1e-12, precision=precision)
    ranks = h.ranks()
    assert ranks[0] >= 10
    if precision == 0:
        o = O.Hodlr(x, "se", th, s2, 64, 1e-12)
        np.testing.assert_array_equal(ranks, o.ranks())
    ll = h.loglik(y)
    sol, ld = O.dense_solve(x, "se", th, s2, y)
    ll_d = -0.5 * y @ sol - 0.5 * ld - 0.5 * n * np.log(2 * np.pi)
    assert abs(ll - ll_d) <= 1e-10 * abs(ll_d), (ll, ll_d)
