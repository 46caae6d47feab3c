"""ORACLE — test infrastructure only. FP64 numpy statement of the rank predictor's network.

The network is not in the paper: a multilayer perceptron x -> tanh(x W1 + b1) ->
tanh(h1 W2 + b2) -> h2 . w3 + b3 with the mean squared error (1/N) sum (y - t)^2, the
parameters flattened as W1 (12 x 64, row-major by input), b1, W2 (64 x 64), b2, w3 (64), b3.
The gradient follows the chain rule written out layer by layer; it is pinned in the tests
by central finite differences.
"""
from __future__ import annotations

import numpy as np

F, Hd = 12, 64
SIZES = [("W1", (F, Hd)), ("b1", (Hd,)), ("W2", (Hd, Hd)), ("b2", (Hd,)), ("w3", (Hd,)), ("b3", (1,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    return out


def forward(p, X):
    q = unpack(p)
    h1 = np.tanh(X @ q["W1"] + q["b1"])
    h2 = np.tanh(h1 @ q["W2"] + q["b2"])
    return h2 @ q["w3"] + q["b3"][0], h1, h2


def loss(p, X, T):
    y, _, _ = forward(p, np.asarray(X, dtype=np.float64))
    return float(np.mean((y - T) ** 2))


def gradient(p, X, T):
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    q = unpack(p)
    y, h1, h2 = forward(p, X)
    n = X.shape[0]
    dy = 2.0 * (y - T) / n                      # d loss / d y
    g_w3 = h2.T @ dy
    g_b3 = np.array([dy.sum()])
    d2 = np.outer(dy, q["w3"]) * (1.0 - h2 ** 2)  # through tanh of layer 2
    g_W2 = h1.T @ d2
    g_b2 = d2.sum(0)
    d1 = (d2 @ q["W2"].T) * (1.0 - h1 ** 2)       # through tanh of layer 1
    g_W1 = X.T @ d1
    g_b1 = d1.sum(0)
    return np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, g_b3])
