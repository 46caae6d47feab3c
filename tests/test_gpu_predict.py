"""GP prediction with the factorization against the dense oracle: posterior mean and latent
variance at test points inside and outside the training range, at training points, in 1-D
and 2-D, both forms; the variance columns are solved in ragged chunks (m = 37)."""
import numpy as np
import pytest

import oracle as O
from paper_1403_6015_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def o2_predict(x, kern, th, s2, y, xt, leaf, max_rank=64):
    """The same prediction through the oracle's HODLR solves (the same approximation)."""
    x2 = x.reshape(len(x), -1)
    xt2 = xt.reshape(len(xt), -1)
    Ks = O.kernel_values(kern, np.sqrt(((x2[:, None, :] - xt2[None, :, :]) ** 2).sum(-1)), th[0], th[1])
    o = O.Hodlr(x, kern, th, s2, leaf, 1e-12, max_rank=max_rank)
    o.factor()
    alpha = o.solve(y)
    V = o.solve(np.asfortranarray(Ks))
    k0 = float(O.kernel_values(kern, np.zeros(1), th[0], th[1])[0])
    return Ks.T @ alpha, k0 - (Ks * V).sum(0)


@pytest.fixture(scope="module")
def H():
    from paper_1403_6015_gb300 import build_lib, hodlr
    build_lib.build()
    hodlr.load()
    return hodlr


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kern,ell", [("matern32", 0.2), ("se", 0.3)])
def test_predict_1d(H, precision, kern, ell):
    n = 4096
    x, y = I.workload_1d(n, 1050)
    xt = np.concatenate([I.uniform_points(30, 1, -1.3, 1.3, 1051), x[::600]])  # m = 37
    th, s2 = [ell, 1.0], 1e-2
    h = H.Hodlr(x, kern, th, s2, 64, 1e-12, precision=precision)
    h.loglik(y)  # factor
    mean, var = h.predict(xt, y)
    # the oracle's HODLR: the same approximation to rounding (FP64 form); the mixed form
    # compresses from double-float entries, a different approximation at eps, so within
    # ~eps cond(C) of it
    m_2, v_2 = o2_predict(x, kern, th, s2, y, xt, 64)
    tol = 1e-10 if precision == 0 else 1e-7
    np.testing.assert_allclose(mean, m_2, rtol=0, atol=tol * np.abs(m_2).max())
    np.testing.assert_allclose(var, v_2, rtol=0, atol=tol)
    # against dense: within the compression error, ~eps cond(C) (cond ~ 1e5 here)
    m_o, v_o = O.dense_predict(x, kern, th, s2, y, xt)
    np.testing.assert_allclose(mean, m_o, rtol=0, atol=1e-7 * np.abs(m_o).max())
    np.testing.assert_allclose(var, v_o, rtol=0, atol=1e-7)
    assert np.all(var >= -1e-7) and np.all(var <= 1.0 + 1e-12)
    # the mean alone, and the factorization is unchanged (a log det read gives the same)
    ld = h.logdet()
    np.testing.assert_array_equal(h.predict(xt, y, var=False), mean)
    assert h.logdet() == ld


def test_predict_2d(H):
    n = 2048
    x, y = I.workload_2d(n, 1052)
    y = np.ascontiguousarray(y).reshape(-1)
    xt = I.uniform_points(21, 2, -0.1, 1.1, 1053)
    th, s2 = [0.3, 1.0], 1e-2
    h = H.Hodlr(x, "matern52", th, s2, 64, 1e-12, max_rank=256)  # 2-D ranks exceed 64
    h.loglik(y)
    mean, var = h.predict(xt, y)
    m_2, v_2 = o2_predict(x, "matern52", th, s2, y, xt, 64, max_rank=256)
    np.testing.assert_allclose(mean, m_2, rtol=0, atol=1e-10 * np.abs(m_2).max())
    np.testing.assert_allclose(var, v_2, rtol=0, atol=1e-10)
    m_o, v_o = O.dense_predict(x, "matern52", th, s2, y, xt)
    np.testing.assert_allclose(mean, m_o, rtol=0, atol=1e-7 * np.abs(m_o).max())
    np.testing.assert_allclose(var, v_o, rtol=0, atol=1e-7)


def test_predict_3d(H):
    n = 2048
    x, y = I.workload_3d(n, 1055)
    y = np.ascontiguousarray(y).reshape(-1)
    xt = I.uniform_points(19, 3, -0.1, 1.1, 1056)
    th, s2 = [0.7, 1.0], 1e-2
    for precision in (0, 1):
        h = H.Hodlr(x, "se", th, s2, 64, 1e-12, max_rank=512, precision=precision)
        h.loglik(y)
        mean, var = h.predict(xt, y)
        m_2, v_2 = o2_predict(x, "se", th, s2, y, xt, 64, max_rank=512)
        tol = 1e-10 if precision == 0 else 1e-7
        np.testing.assert_allclose(mean, m_2, rtol=0, atol=tol * np.abs(m_2).max())
        np.testing.assert_allclose(var, v_2, rtol=0, atol=tol)
        m_o, v_o = O.dense_predict(x, "se", th, s2, y, xt)
        np.testing.assert_allclose(mean, m_o, rtol=0, atol=1e-7 * np.abs(m_o).max())
        np.testing.assert_allclose(var, v_o, rtol=0, atol=1e-7)


def test_predict_needs_a_factor(H):
    x, y = I.workload_1d(1024, 1054)
    h = H.Hodlr(x, "exp", [0.2, 1.0], 1e-2, 64, 1e-12)
    with pytest.raises(H.HodlrError):
        h.predict(x[:3], y)
