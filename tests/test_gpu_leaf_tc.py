"""The tensor-core leaf kernel of the mixed form (leaf_kernel = 1: trailing updates and
off-diagonal solve updates as exact bf16-slice products on tcgen05, the rest in
double-float) against the CPU oracle, with the same bars as the FP32-pipe leaf kernel:
log det and log-likelihood within 1e-10 relative, solutions within 1e-9 of the largest
entry, exact residual rows within 1e-10 at the full size."""
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


def tc_context(H, x, kern, th, s2, leaf, eps, **kw):
    h = H.Hodlr(x, kern, th, s2, leaf, eps, precision=1, **kw)
    h.set_tuning(512, 0, 1)
    assert h.tuning()["leaf_kernel"] == 1
    h.rebuild(th, s2)
    return h


# leaves of 1 .. 128 points: one, two, three and four 32-column panels, ragged tails
@pytest.mark.parametrize("n,leaf", [(1, 8), (33, 64), (100, 7), (1000, 64), (3000, 100),
                                    (4096, 128), (10000, 97)])
@pytest.mark.parametrize("kern", ["exp", "se", "matern32", "matern52"])
def test_tc_leaf_vs_oracle(H, n, leaf, kern):
    x, y = I.workload_1d(n, 800 + n, nrhs=2)
    th, s2 = [0.3, 1.2], 0.05
    h = tc_context(H, x, kern, th, s2, leaf, 1e-13)
    sol = h.factor_solve(y)
    ref = O.Hodlr(x, kern, th, s2, leaf, 1e-13)
    sol_o = ref.factor_solve(y)
    assert abs(h.logdet() - ref.logdet()) <= 1e-10 * max(1.0, abs(ref.logdet()))
    np.testing.assert_allclose(sol, sol_o, rtol=0, atol=1e-9 * np.abs(sol_o).max())


def test_tc_leaf_many_columns(H):
    """More panel and right-hand-side columns than one 32-column solve chunk (three
    chunks), 2-D points."""
    n = 6000
    x, y = I.workload_2d(n, 94, nrhs=16)
    th, s2 = [0.3, 1.0], 0.01
    h = tc_context(H, x, "se", th, s2, 128, 1e-10, max_rank=128)
    sol = h.factor_solve(y)
    assert sum(h.level_ranks()) + 16 > 64
    ref = O.Hodlr(x, "se", th, s2, 128, 1e-10, max_rank=128)
    sol_o = ref.factor_solve(y)
    assert rel(h.logdet(), ref.logdet()) <= 1e-10
    np.testing.assert_allclose(sol, sol_o, rtol=0, atol=1e-9 * np.abs(sol_o).max())


def test_tc_leaf_dense_small(H):
    """One leaf: the whole matrix is the dense leaf block, against dense Cholesky."""
    x, y = I.workload_1d(128, 95)
    th, s2 = [0.5, 1.0], 1e-3
    h = tc_context(H, x, "se", th, s2, 128, 1e-12)
    sol = h.factor_solve(y)
    sol_d, ld_d = O.dense_solve(x, "se", th, s2, y)
    assert rel(h.logdet(), ld_d) <= 1e-10
    np.testing.assert_allclose(sol, sol_d, rtol=0, atol=1e-9 * np.abs(sol_d).max())


@pytest.mark.parametrize("kern,ell", [("matern32", 0.1), ("exp", 0.2)])
def test_tc_leaf_full_size(H, kern, ell):
    """n = 2^20, sigma^2 = 1e-2, leaf 128, eps = 1e-12 (the bench's workload) against the
    exact O(n) oracles: log det, log-likelihood and exact residual rows."""
    n = 1 << 20
    x, y = I.workload_1d(n, 1002)
    s2 = 1e-2
    h = tc_context(H, x, kern, [ell, 1.0], s2, 128, 1e-12)
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


def test_tc_leaf_flags_not_spd(H):
    x = np.linspace(-1, 1, 64)
    x[1] = x[0]
    h = H.Hodlr(x, "se", [0.3, 1.0], 0.0, 64, 1e-12, precision=1)
    h.set_tuning(512, 0, 1)
    with pytest.raises(H.HodlrError) as e:
        h.factor()
    assert e.value.status == H.HODLR_ENOTSPD
