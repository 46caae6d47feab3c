"""3-D points. The method does not depend on the dimension (Sec. 3 orders the points by a
recursive split and compresses the off-diagonal blocks whatever their geometry); what
changes is the kd ordering, which cycles through three coordinates, the Euclidean
distance over three, and the block ranks, which grow with the dimension (here 100-340 at
n = 3000). Checked against the oracle (ordering bit-exact, ranks, log det, solution) and
dense Cholesky, in both precisions."""
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


def level_max(ranks, kappa):
    return np.array([ranks[(1 << j) - 1:(1 << (j + 1)) - 1].max() for j in range(kappa)])


@pytest.mark.parametrize("n,leaf", [(50, 8), (3001, 20), (1 << 15, 64)])
def test_sort_3d_kd_bit_exact(H, n, leaf):
    x, _ = I.workload_3d(n, 17 + n)
    h = H.Hodlr(x, "se", [1.0, 1.0], 0.01, leaf, 1e-6, allow_rank_cap=True)
    _, perm = h.tree()
    np.testing.assert_array_equal(perm, O.tree_order(x, leaf))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kern,ell,eps,ld_tol", [("se", 0.5, 1e-12, 1e-12),
                                                 ("matern52", 2.0, 1e-10, 1e-10)])
def test_3d_vs_oracle_and_dense(H, kern, ell, eps, ld_tol, precision):
    """Top-level ranks above 300: the blocked node step and the sweep in product form."""
    n = 3000
    x, y = I.workload_3d(n, 94)
    y = np.ascontiguousarray(y).reshape(-1)
    th, s2 = [ell, 1.0], 0.01
    h = H.Hodlr(x, kern, th, s2, 32, eps, max_rank=512, precision=precision)
    sol = h.factor_solve(y)
    ld = h.logdet()
    o = O.Hodlr(x, kern, th, s2, 32, eps, max_rank=512)
    sol_o = o.factor_solve(y)
    ld_o = o.logdet()
    kappa, _ = h.tree()
    lv, lv_o = level_max(h.ranks(), kappa), level_max(o.ranks(), o.kappa)
    assert lv[0] > 300
    # the ACA's terms decay slowly near eps here, so the rounding of the mixed form's
    # entries can move its stop by a few steps without changing the accuracy
    assert np.all(np.abs(lv - lv_o) <= np.maximum(2, 0.03 * lv_o)), (lv, lv_o)
    sol_d, ld_d = O.dense_solve(x, kern, th, s2, y)
    print(f"{kern} prec {precision}: ranks {lv.tolist()} logdet vs oracle {rel(ld, ld_o):.2e} "
          f"vs dense {rel(ld, ld_d):.2e}")
    assert rel(ld, ld_o) <= (1e-12 if precision == 0 else 1e-11)
    assert rel(ld, ld_d) <= ld_tol + 1e-12
    # the factorization solves its own compressed operator to rounding (the mixed form's
    # panels carry 48-bit significands), and the solution is as close to C^-1 y as the
    # oracle's
    res_own = np.linalg.norm(y - h.matvec(sol)) / np.linalg.norm(y)
    assert res_own <= (3e-11 if precision == 0 else 3e-10), res_own
    err, err_o = np.abs(sol - sol_d).max(), np.abs(sol_o - sol_d).max()
    assert err <= 4.0 * err_o + 1e-12 * np.abs(sol_d).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_3d_loglik_n2p15(H, precision):
    n = 1 << 15
    x, y = I.workload_3d(n, 95)
    y = np.ascontiguousarray(y).reshape(-1)
    th, s2 = [1.0, 1.0], 0.01
    h = H.Hodlr(x, "se", th, s2, 64, 1e-10, max_rank=256, precision=precision)
    ll = h.loglik(y)
    ll_o = O.Hodlr(x, "se", th, s2, 64, 1e-10, max_rank=256).loglik(y)
    assert rel(ll, ll_o) <= 1e-10, (ll, ll_o)


def test_3d_default_rank_cap_reports(H):
    """A 3-D Matern-3/2 problem whose top block needs more than the default cap of 64: the
    build reports the rank cap rather than returning a silently truncated factor."""
    x, _ = I.workload_3d(3000, 96)
    with pytest.raises(H.HodlrError):
        H.Hodlr(x, "matern32", [1.0, 1.0], 0.01, 32, 1e-10)


@pytest.mark.parametrize("precision", [0, 1])
def test_3d_ranks_above_512(H, precision):
    """3-D Matern-3/2 (ell = 1, eps = 1e-10): top-level ranks above 600, under the cap of
    1024; the node matrices of those levels (2r > 1200) are factored in global memory."""
    n = 3000
    x, y = I.workload_3d(n, 97)
    y = np.ascontiguousarray(y).reshape(-1)
    th, s2 = [1.0, 1.0], 0.01
    h = H.Hodlr(x, "matern32", th, s2, 32, 1e-10, max_rank=1024, precision=precision)
    sol = h.factor_solve(y)
    ld = h.logdet()
    o = O.Hodlr(x, "matern32", th, s2, 32, 1e-10, max_rank=1024)
    o.factor_solve(y)
    kappa, _ = h.tree()
    lv, lv_o = level_max(h.ranks(), kappa), level_max(o.ranks(), o.kappa)
    assert lv[0] > 512
    assert np.all(np.abs(lv - lv_o) <= np.maximum(2, 0.03 * lv_o)), (lv, lv_o)
    _, ld_d = O.dense_solve(x, "matern32", th, s2, y)
    print(f"matern32 3-D prec {precision}: ranks {lv.tolist()} logdet vs oracle "
          f"{rel(ld, o.logdet()):.2e} vs dense {rel(ld, ld_d):.2e}")
    assert rel(ld, o.logdet()) <= (1e-12 if precision == 0 else 1e-11)
    assert rel(ld, ld_d) <= 1e-10
    res_own = np.linalg.norm(y - h.matvec(sol)) / np.linalg.norm(y)
    assert res_own <= (3e-11 if precision == 0 else 3e-10), res_own
