"""Chebyshev interpolation compression on the GPU (Sec. 3.1's analytic A ~ E A~ P),
against the oracle's Chebyshev HODLR (same approximation), dense factorizations, and at
the full size n = 2^20 against the Ornstein-Uhlenbeck closed form and the Kalman filter."""
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


@pytest.mark.parametrize("kern,rank", [("exp", 1), ("matern32", 2), ("matern52", 3)])
@pytest.mark.parametrize("precision", [0, 1])
def test_exact_ranks(H, kern, rank, precision):
    x, _ = I.workload_1d(20000, 61)
    h = H.Hodlr(x, kern, [0.1, 1.0], 0.01, 64, 1e-10, precision=precision,
                compression="chebyshev")
    assert np.all(h.ranks() == rank)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kern,ell,s2,n,leaf", [("se", 0.3, 0.01, 20000, 100),
                                                ("matern52", 0.2, 0.01, 12345, 64),
                                                ("imq", 0.5, 1.0, 9000, 37),
                                                ("rq", 0.8, 1.0, 5000, 128),
                                                ("mq", 1.0, 1.0, 7000, 50)])
def test_vs_oracle(H, kern, ell, s2, n, leaf, precision):
    if kern in H.INDEFINITE and precision == 1:
        pytest.skip("indefinite kernels need the FP64 form")
    x, y = I.workload_1d(n, 62 + n, lo=-3.0, hi=3.0)
    h = H.Hodlr(x, kern, [ell, 1.0], s2, leaf, 1e-12, max_rank=256, precision=precision,
                compression="chebyshev")
    sol = h.factor_solve(y)
    o = O.Hodlr(x, kern, [ell, 1.0], s2, leaf, 1e-12, max_rank=256, compression="chebyshev")
    sol_o = o.factor_solve(y)
    lad, sg = h.logdet_signed()
    dr = np.abs(h.ranks() - o.ranks()).max()
    print(f"{kern} prec {precision}: max rank {h.ranks().max()} (oracle {o.ranks().max()}, "
          f"largest difference {dr}), log|det| vs oracle {rel(lad, o.logdet()):.2e}")
    assert dr <= 1
    assert sg == o.logdet_sign()
    assert rel(lad, o.logdet()) <= (1e-12 if precision == 0 else 1e-11)
    np.testing.assert_allclose(sol, sol_o, rtol=0, atol=1e-9 * np.abs(sol_o).max())


def test_vs_dense_and_aca(H):
    n = 3000
    x, y = I.workload_1d(n, 63, lo=-3.0, hi=3.0)
    x[101] = x[100]  # a duplicated point
    th, s2 = [0.5, 1.0], 0.01
    sol_d, ld_d = O.dense_solve(x, "se", th, s2, y)
    hc = H.Hodlr(x, "se", th, s2, 32, 1e-12, compression="chebyshev")
    ha = H.Hodlr(x, "se", th, s2, 32, 1e-12)
    sc, sa = hc.factor_solve(y), ha.factor_solve(y)
    assert rel(hc.logdet(), ld_d) <= 1e-12
    assert rel(hc.logdet(), ha.logdet()) <= 1e-12
    np.testing.assert_allclose(sc, sol_d, rtol=0, atol=1e-8 * np.abs(sol_d).max())


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_closed_forms(H, precision):
    """n = 2^20, the exponential kernel against the OU closed form (log det and the whole
    solution) and Matern-3/2 against the Kalman filter (log det and y^T C^-1 y)."""
    n = 1 << 20
    x, y = I.workload_1d(n, 1000)
    perm = np.argsort(x[:, 0], kind="stable")
    xs, ys = x[perm, 0], y[perm]
    h = H.Hodlr(x, "exp", [0.2, 1.0], 0.05, 128, 1e-12, precision=precision,
                compression="chebyshev")
    sol = h.factor_solve(y)
    sol_ou, ld_ou = O.ou_closed_form(xs, 0.2, 1.0, 0.05, ys)
    assert rel(h.logdet(), ld_ou) <= 1e-10
    # the bar of the cross approximation's own full-size test
    assert np.linalg.norm(sol[perm] - sol_ou) <= 1e-9 * np.linalg.norm(sol_ou)
    h = H.Hodlr(x, "matern32", [0.3, 1.0], 0.05, 128, 1e-12, precision=precision,
                compression="chebyshev")
    ll = h.loglik(y)
    ld_k, q_k = O.matern_kalman(xs, 3, 0.3, 1.0, 0.05, ys)
    ll_k = -0.5 * q_k - 0.5 * ld_k - 0.5 * n * np.log(2 * np.pi)
    assert rel(ll, ll_k) <= 1e-10
    assert rel(h.logdet(), ld_k) <= 1e-10


def test_reports_and_refusals(H):
    x, y = I.workload_1d(2000, 64, lo=-3.0, hi=3.0)
    st, ctx = H.hodlr_build(x, 2000, 1, H.KERNELS["biharmonic"], [1.0, 1.0], 2.0, 32, 1e-12,
                            _opts(H, compression=1))
    assert st == H.HODLR_ERANK  # r^2 log r is not smooth where the clusters meet
    H.hodlr_destroy(ctx)
    h = H.Hodlr(x, "se", [0.5, 1.0], 0.01, 32, 1e-12, compression="chebyshev")
    with pytest.raises(H.HodlrError):
        h.presize(np.full(h.tree()[0], 8, dtype=np.int32))


def test_leaf_one_empty_children(H):
    """Leaf size 1 leaves some children empty: their blocks are exact at rank 0."""
    for n in (3, 5, 6, 11):
        x, y = I.workload_1d(n, 65 + n)
        sol_d, ld_d = O.dense_solve(x, "se", [0.5, 1.0], 0.1, y)
        h = H.Hodlr(x, "se", [0.5, 1.0], 0.1, 1, 1e-13, compression="chebyshev")
        sol = h.factor_solve(y)
        assert abs(h.logdet() - ld_d) <= 1e-12 * max(1.0, abs(ld_d))
        np.testing.assert_allclose(sol, sol_d, rtol=0, atol=1e-11 * np.abs(sol_d).max())


def _opts(H, **kw):
    o = H.hodlr_default_opts()
    for k, v in kw.items():
        setattr(o, k, v)
    return o
