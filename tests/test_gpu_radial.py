"""The radial functions of Sec. 5 on the GPU: rational quadratic and inverse multiquadric
(positive definite: the regular path, both precisions, log-likelihood) and the indefinite
multiquadric and biharmonic (LU leaves with partial pivoting, signed log |det|, no
log-likelihood). Checked against the oracle's HODLR (same approximation), its dense LU or
Cholesky (the definition), and LAPACK through numpy. Workloads follow Sec. 5's tables:
points uniform in [-3, 3]^d, C = I + K (multiquadric, inverse multiquadric) or 2I + K
(biharmonic)."""
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


def pts(n, d, seed):
    return I.uniform_points(n, d, -3.0, 3.0, seed), I.normal(n, seed + 1)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kern,theta,d", [("imq", [1.0, 1.0], 1), ("rq", [0.5, 1.3, 2.0], 1),
                                          ("rq", [0.8, 1.0, 0.7], 2), ("imq", [0.5, 1.0], 2)])
def test_positive_radial_vs_oracle(H, kern, theta, d, precision):
    n = 3000 if d == 1 else 2000
    x, y = pts(n, d, 2000 + 10 * d)
    alpha = theta[2] if len(theta) > 2 else 1.0
    h = H.Hodlr(x, kern, theta[:2], 1.0, 32, 1e-12, max_rank=512, precision=precision,
                rq_alpha=alpha)
    sol = h.factor_solve(y)
    ld = h.logdet()
    o = O.Hodlr(x, kern, theta, 1.0, 32, 1e-12, max_rank=512)
    sol_o = o.factor_solve(y)
    sol_d, ld_d = O.dense_solve(x, kern, theta, 1.0, y)
    print(f"{kern} d{d} prec {precision}: logdet vs oracle {rel(ld, o.logdet()):.2e} vs dense "
          f"{rel(ld, ld_d):.2e}; ranks {h.ranks().max()}")
    assert rel(ld, o.logdet()) <= 1e-12
    assert rel(ld, ld_d) <= 1e-11
    np.testing.assert_allclose(sol, sol_o, rtol=0, atol=1e-10 * np.abs(sol_o).max())
    assert h.logdet_signed() == (ld, 1)
    ll = H.Hodlr(x, kern, theta[:2], 1.0, 32, 1e-12, max_rank=512, precision=precision,
                 rq_alpha=alpha).loglik(y)
    assert rel(ll, o.loglik(y)) <= 1e-12


@pytest.mark.parametrize("kern,d,s2,eps", [("mq", 1, 1.0, 1e-12), ("biharmonic", 1, 2.0, 1e-12),
                                           ("mq", 2, 1.0, 1e-14), ("biharmonic", 2, 2.0, 1e-12)])
def test_indefinite_vs_oracle_and_dense(H, kern, d, s2, eps):
    n = 2000
    x, y = pts(n, d, 2100 + 10 * d)
    h = H.Hodlr(x, kern, [1.0, 1.0], s2, 32, eps, max_rank=512)
    sol = h.factor_solve(y)
    lad, sg = h.logdet_signed()
    o = O.Hodlr(x, kern, [1.0, 1.0], s2, 32, eps, max_rank=512)
    sol_o = o.factor_solve(y)
    sol_d, ld_d, sg_d = O.dense_lu_solve(x, kern, [1.0, 1.0], s2, y)
    print(f"{kern} d{d}: sign {sg} (dense {sg_d}), log|det| vs oracle {rel(lad, o.logdet()):.2e} "
          f"vs dense {rel(lad, ld_d):.2e}; ranks {h.ranks().max()}")
    assert sg == sg_d == o.logdet_sign()
    assert rel(lad, o.logdet()) <= 1e-12
    assert rel(lad, ld_d) <= 1e-10
    assert h.logdet() == lad
    np.testing.assert_allclose(sol, sol_o, rtol=0, atol=1e-9 * np.abs(sol_o).max())
    np.testing.assert_allclose(sol, sol_d, rtol=0, atol=1e-8 * np.abs(sol_d).max())
    # a second solve with the stored factor (the LU row orders read back)
    y2 = I.normal(n, 2199)
    np.testing.assert_allclose(h.solve(y2), o.solve(y2), rtol=0,
                               atol=1e-9 * np.abs(o.solve(y2)).max())


@pytest.mark.parametrize("n,leaf", [(1, 8), (100, 128), (128, 128), (1000, 37), (4097, 64)])
def test_multiquadric_ragged_and_single_leaf(H, n, leaf):
    """Single-leaf problems factor the whole C by the leaf LU (pivoting over up to 128
    rows); ragged leaves exercise the pivot search on partial blocks."""
    x, y = pts(n, 1, 2200 + n)
    sol_d, ld_d, sg_d = O.dense_lu_solve(x, "mq", [1.0, 1.0], 1.0, y)
    h = H.Hodlr(x, "mq", [1.0, 1.0], 1.0, leaf, 1e-13, max_rank=512)
    sol = h.factor_solve(y)
    lad, sg = h.logdet_signed()
    assert sg == sg_d
    assert abs(lad - ld_d) <= 1e-11 * max(1.0, abs(ld_d))
    np.testing.assert_allclose(sol, sol_d, rtol=0, atol=1e-9 * np.abs(sol_d).max())


def test_both_signs_occur(H):
    """det C changes sign with the number of negative eigenvalues of C = s2 I + K; over
    these sizes both signs occur, and each matches dense LU."""
    seen = set()
    for n in (300, 301, 302, 303, 500, 777):
        x, _ = pts(n, 1, 2300 + n)
        _, _, sg_d = O.dense_lu_solve(x, "mq", [1.0, 1.0], 1.0, np.ones(n))
        h = H.Hodlr(x, "mq", [1.0, 1.0], 1.0, 16, 1e-12, max_rank=512)
        h.factor()
        assert h.logdet_signed()[1] == sg_d, n
        seen.add(sg_d)
    assert seen == {1, -1}


def test_indefinite_refinement(H):
    x, y = pts(8192, 1, 2400)
    h = H.Hodlr(x, "biharmonic", [1.0, 1.0], 2.0, 64, 1e-10, max_rank=512, refine_maxit=3,
                refine_tol=1e-13)
    sol = h.factor_solve(y)
    corr, res = h.refine_info()
    assert corr >= 1 and res <= 1e-13
    np.testing.assert_allclose(h.matvec(sol), y, rtol=0, atol=1e-12 * np.abs(y).max())
    o = O.Hodlr(x, "biharmonic", [1.0, 1.0], 2.0, 64, 1e-10, max_rank=512)
    o.factor()
    assert h.logdet_signed()[1] == o.logdet_sign()


def test_indefinite_refusals(H):
    x, y = pts(1000, 1, 2500)
    h = H.Hodlr(x, "mq", [1.0, 1.0], 1.0, 32, 1e-12)
    with pytest.raises(H.HodlrError):
        h.loglik(y)  # C is not a covariance
    with pytest.raises(H.HodlrError):
        h.presize(np.full(h.tree()[0], 8, dtype=np.int32))
    with pytest.raises(H.HodlrError):
        H.Hodlr(x, "biharmonic", [1.0, 1.0], 2.0, 32, 1e-12, precision=1)


def test_imq_interpolation_prediction(H):
    """The posterior mean with an inverse multiquadric covariance is the kriging
    interpolant; against the dense formula."""
    n = 2048
    x, y = pts(n, 1, 2600)
    xt = I.uniform_points(23, 1, -3.2, 3.2, 2601)
    for precision in (0, 1):
        h = H.Hodlr(x, "imq", [0.4, 1.0], 0.1, 64, 1e-12, precision=precision)
        h.loglik(y)
        mean, var = h.predict(xt, y)
        m_o, v_o = O.dense_predict(x, "imq", [0.4, 1.0], 0.1, y, xt)
        np.testing.assert_allclose(mean, m_o, rtol=0, atol=1e-8 * np.abs(m_o).max())
        np.testing.assert_allclose(var, v_o, rtol=0, atol=1e-8)
