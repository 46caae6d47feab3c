"""The paper's regression experiment (Sec. 5.7) on synthetic data of the same model: 1024
points x ~ U(-3, 3), y = sin(2x) + e^x / 8 + noise (sigma = 1), kernel exp(-(x - x')^2),
leaf 20; the regression estimate at the data points y_hat = K (sigma^2 I + K)^-1 y (the
posterior mean there) through the factorization against dense linear algebra: the RMSE
difference falls with the factorization precision eps, roughly in proportion."""
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


def test_rmse_difference_proportional_to_eps(H):
    n = 1024
    x = I.uniform_points(n, 1, -3.0, 3.0, 1060)[:, 0]
    y = np.sin(2 * x) + np.exp(x) / 8 + I.normal(n, 1061)
    th, s2 = [0.5 ** 0.5, 1.0], 1.0  # exp(-(x - x')^2) = exp(-r^2 / (2 ell^2))
    mean_d, _ = O.dense_predict(x, "se", th, s2, y, x)
    rmse_d = np.linalg.norm(y - mean_d) / np.sqrt(n)
    diffs = []
    epss = [1e-2, 1e-4, 1e-6, 1e-8, 1e-10, 1e-12]
    for eps in epss:
        h = H.Hodlr(x, "se", th, s2, 20, eps)
        h.loglik(y)
        mean = h.predict(x, y, var=False)
        diffs.append(abs(np.linalg.norm(y - mean) / np.sqrt(n) - rmse_d))
    print("dense RMSE %.16f; |RMSE - dense RMSE| by eps:" % rmse_d,
          ", ".join("%.0e: %.2e" % (e, d) for e, d in zip(epss, diffs)))
    assert 0.5 < rmse_d < 1.5  # noise of unit variance
    for e, d in zip(epss, diffs):
        assert d <= 10 * e
    assert diffs[-1] < diffs[0]
