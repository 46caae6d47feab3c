"""Pins for the FP64 oracle of the rank predictor's network: its analytic gradient against
central finite differences of its loss (a plausible slip in any layer's chain rule, a
missing tanh derivative or a transposed weight, fails this)."""
import numpy as np

from oracle import mlp_oracle as M


def test_param_count():
    assert M.NPARAMS == 12 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 5057


def test_gradient_vs_finite_differences():
    rng = np.random.default_rng(3)
    p = rng.standard_normal(M.NPARAMS) * 0.2
    X = rng.standard_normal((40, 12))
    T = rng.standard_normal(40)
    g = M.gradient(p, X, T)
    h = 1e-6
    idx = np.concatenate([rng.choice(M.NPARAMS, 200, replace=False), [M.NPARAMS - 1, 0, 768]])
    for i in idx:
        e = np.zeros(M.NPARAMS)
        e[i] = h
        fd = (M.loss(p + e, X, T) - M.loss(p - e, X, T)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_forward_shapes_and_bias():
    p = np.zeros(M.NPARAMS)
    p[-1] = 0.75
    y, h1, h2 = M.forward(p, np.ones((3, 12)))
    np.testing.assert_allclose(y, 0.75)
    assert h1.shape == (3, 64) and h2.shape == (3, 64)
