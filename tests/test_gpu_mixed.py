"""Parity of the mixed-precision form (double-float leaf stage, FP64 elsewhere) with the
FP64 oracle. The same bars as the FP64 form: log det and log-likelihood within 1e-10
relative, residuals within the oracle's own residual scale."""
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


def rel(a, b):
    return abs(a - b) / abs(b)


@pytest.mark.parametrize("n,leaf", [(1, 8), (9, 8), (100, 7), (1000, 64), (3000, 128), (10000, 100)])
@pytest.mark.parametrize("kern", ["exp", "se", "matern32", "matern52"])
def test_mixed_vs_oracle(H, n, leaf, kern):
    x, y = I.workload_1d(n, 700 + n, nrhs=2)
    th, s2 = [0.3, 1.2], 0.05
    h = H.Hodlr(x, kern, th, s2, leaf, 1e-13, precision=1)
    sol = h.factor_solve(y)
    ref = O.Hodlr(x, kern, th, s2, leaf, 1e-13)
    sol_o = ref.factor_solve(y)
    assert abs(h.logdet() - ref.logdet()) <= 1e-10 * max(1.0, abs(ref.logdet()))
    np.testing.assert_allclose(sol, sol_o, rtol=0, atol=1e-9 * np.abs(sol_o).max())


def test_mixed_2d(H):
    n = 3000
    x, y = I.workload_2d(n, 93)
    th, s2 = [0.5, 1.0], 0.01
    h = H.Hodlr(x, "se", th, s2, 32, 1e-12, precision=1)
    h.factor_solve(y)
    ref = O.Hodlr(x, "se", th, s2, 32, 1e-12)
    ref.factor()
    assert rel(h.logdet(), ref.logdet()) <= 1e-10


def test_mixed_standalone_solve(H):
    x, y = I.workload_1d(5000, 44, nrhs=3)
    h = H.Hodlr(x, "matern52", [0.2, 1.0], 0.01, 64, 1e-12, precision=1)
    h.factor()
    sol = h.solve(y)
    ref = O.Hodlr(x, "matern52", [0.2, 1.0], 0.01, 64, 1e-12)
    ref.factor()
    sol_o = ref.solve(y)
    np.testing.assert_allclose(sol, sol_o, rtol=0, atol=1e-9 * np.abs(sol_o).max())


@pytest.mark.parametrize("kern,ell", [("matern32", 0.1), ("exp", 0.2)])
def test_mixed_full_size(H, kern, ell):
    """n = 2^20, sigma^2 = 1e-2, leaf 128, eps = 1e-12 (the bench's workload) against the
    exact O(n) oracles: log det, log-likelihood and exact residual rows."""
    n = 1 << 20
    x, y = I.workload_1d(n, 1002)
    s2 = 1e-2
    h = H.Hodlr(x, kern, [ell, 1.0], s2, 128, 1e-12, precision=1)
    ll = h.loglik(y)
    h.rebuild([ell, 1.0], s2)
    sol = h.factor_solve(y)
    _, perm = h.tree()
    if kern == "exp":
        sol_c, ld_c = O.ou_closed_form(x[perm, 0], ell, 1.0, s2, y[perm])
        q_c = float(y[perm] @ sol_c)
    else:
        ld_c, q_c = O.matern_kalman(x[perm, 0], 3, ell, 1.0, s2, y[perm])
    ll_c = -0.5 * q_c - 0.5 * ld_c - 0.5 * n * np.log(2 * np.pi)
    assert rel(h.logdet(), ld_c) <= 1e-10
    assert rel(ll, ll_c) <= 1e-10
    rows = np.unique(np.linspace(0, n - 1, 64).astype(np.int64))
    Cx = O.dense_matvec_rows(x, kern, [ell, 1.0], s2, sol, rows)
    assert np.abs(Cx - y[rows]).max() / np.abs(y).max() <= 1e-10
