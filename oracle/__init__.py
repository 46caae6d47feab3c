"""ORACLE loader — test infrastructure only.

ctypes binding of the plain FP64 CPU oracle in hodlr_oracle.c. Only tests/,
__graft_entry__.smoke() and bench.py's CPU-baseline leg may import this package; the
CUDA library never does, and this package never imports the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hodlr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

KERNELS = {"exp": 0, "se": 1, "matern32": 2, "matern52": 3, "rq": 4, "imq": 5, "mq": 6,
           "biharmonic": 7}
# Kernels whose matrices are indefinite: factor, solve and log |det| with its sign, no
# log-likelihood.
INDEFINITE = ("mq", "biharmonic")
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ENOTSPD", 4: "ERANK", 6: "ESTATE"}

_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc: -O2, no FMA contraction (same rounding on x86 and Arm), OpenMP."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.oracle_num_threads.restype = ctypes.c_int
        L.oracle_set_num_threads.argtypes = [ctypes.c_int]
        L.oracle_kernel_values.argtypes = [ctypes.c_int, _dp, ctypes.c_int64, _dp, _dp]
        L.oracle_dense_lu_solve.argtypes = [_dp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _dp,
                                            ctypes.c_double, _dp, ctypes.c_int, ctypes.c_int64, _dp,
                                            ctypes.c_int64, _dp, _ip]
        L.oracle_dense_solve.argtypes = [_dp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _dp,
                                         ctypes.c_double, _dp, ctypes.c_int, ctypes.c_int64, _dp,
                                         ctypes.c_int64, _dp]
        L.oracle_dense_matvec_rows.argtypes = [_dp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _dp,
                                               ctypes.c_double, _dp, _lp, ctypes.c_int64, _dp]
        L.oracle_ou_closed_form.argtypes = [_dp, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, _dp, ctypes.c_int, ctypes.c_int64, _dp,
                                            ctypes.c_int64, _dp]
        L.oracle_matern_kalman.argtypes = [_dp, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, _dp, _dp, _dp]
        L.oracle_lu_logdet.argtypes = [_dp, ctypes.c_int, _ip]
        L.oracle_lu_logdet.restype = ctypes.c_double
        L.oracle_lu_solve_dense.argtypes = [_dp, ctypes.c_int, _dp, _dp]
        L.oracle_kappa.argtypes = [ctypes.c_int64, ctypes.c_int]
        L.oracle_kappa.restype = ctypes.c_int
        L.oracle_tree_order.argtypes = [_dp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _lp]
        L.oracle_hodlr_build.argtypes = [_dp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _dp,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_int, ctypes.c_int, _ip]
        L.oracle_hodlr_build.restype = ctypes.c_void_p
        L.oracle_hodlr_kappa.argtypes = [ctypes.c_void_p]
        L.oracle_hodlr_kappa.restype = ctypes.c_int
        L.oracle_hodlr_ranks.argtypes = [ctypes.c_void_p, _ip, ctypes.c_int64]
        L.oracle_hodlr_ranks.restype = ctypes.c_int64
        L.oracle_hodlr_perm.argtypes = [ctypes.c_void_p, _lp]
        L.oracle_hodlr_factor.argtypes = [ctypes.c_void_p]
        L.oracle_hodlr_solve.argtypes = [ctypes.c_void_p, _dp, _dp, ctypes.c_int, ctypes.c_int64]
        L.oracle_hodlr_factor_solve.argtypes = [ctypes.c_void_p, _dp, _dp, ctypes.c_int,
                                                ctypes.c_int64]
        L.oracle_hodlr_logdet.argtypes = [ctypes.c_void_p, _dp]
        L.oracle_hodlr_logdet_sign.argtypes = [ctypes.c_void_p, _ip]
        L.oracle_hodlr_level_logdets.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.oracle_hodlr_loglik.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.oracle_hodlr_matvec.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.oracle_hodlr_node_factors.argtypes = [ctypes.c_void_p, ctypes.c_int64, _dp, _dp]
        L.oracle_hodlr_node_factors.restype = ctypes.c_int
        L.oracle_hodlr_node_range.argtypes = [ctypes.c_void_p, ctypes.c_int64, _lp, _lp]
        L.oracle_hodlr_destroy.argtypes = [ctypes.c_void_p]
        _lib = L
    return _lib


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    pass


def _check(st: int, what: str):
    if st != 0:
        raise OracleError(f"{what}: status {STATUS.get(st, st)}")


def num_threads() -> int:
    return lib().oracle_num_threads()


def set_num_threads(t: int) -> None:
    """Threads of the oracle's OpenMP loops (t < 1: all host cores); results do not depend
    on it."""
    lib().oracle_set_num_threads(int(t))


def _theta(theta) -> np.ndarray:
    """{ell, a} or {ell, a, alpha} (alpha: the rational quadratic's exponent, default 1)."""
    th = np.ones(3)
    t = np.asarray(theta, dtype=np.float64).reshape(-1)
    th[: t.size] = t
    return th


def kernel_values(kernel: str, r, ell: float, amp: float = 1.0, alpha: float = 1.0) -> np.ndarray:
    r = _f64(r)
    out = np.empty_like(r)
    th = _theta([ell, amp, alpha])
    lib().oracle_kernel_values(KERNELS[kernel], _d(r), r.size, _d(th), _d(out))
    return out


def _cols(y):
    y = np.asarray(y, dtype=np.float64)
    one = y.ndim == 1
    Y = np.asfortranarray(y.reshape(-1, 1) if one else y)
    return Y, one


def dense_solve(x, kernel, theta, sigma2, y):
    """O1: (C^-1 y, log det C) by dense Cholesky; y (n,) or (n, nrhs)."""
    x = _f64(x)
    n, d = (x.shape[0], 1) if x.ndim == 1 else x.shape
    Y, one = _cols(y)
    X = np.zeros_like(Y, order="F")
    ld = ctypes.c_double()
    th = _theta(theta)
    _check(lib().oracle_dense_solve(_d(x), n, d, KERNELS[kernel], _d(th), sigma2, _d(Y), Y.shape[1],
                                    n, _d(X), n, ctypes.byref(ld)), "dense_solve")
    return (X[:, 0] if one else X), ld.value


def dense_predict(x, kernel, theta, sigma2, y, xtest):
    """GP prediction from the dense factorization (O1): the posterior mean k_*^T C^-1 y
    and the latent posterior variance k(x*, x*) - k_*^T C^-1 k_* at each test point (the
    conditional distribution behind the likelihood of Sec. 1; the standard GP regression
    formulas). x: (n, d) or (n,), xtest: (m, d) or (m,). Returns (mean, var), each (m,)."""
    x = _f64(x).reshape(len(x), -1)
    xt = _f64(xtest).reshape(len(xtest), -1)
    r = np.sqrt(((x[:, None, :] - xt[None, :, :]) ** 2).sum(-1))
    th = _theta(theta)
    Ks = kernel_values(kernel, r, *th)  # n x m
    w, _ = dense_solve(x, kernel, th, sigma2, y)
    V, _ = dense_solve(x, kernel, th, sigma2, np.asfortranarray(Ks))
    mean = Ks.T @ w
    var = float(kernel_values(kernel, np.zeros(1), *th)[0]) - (Ks * V).sum(0)
    return mean, var


def dense_lu_solve(x, kernel, theta, sigma2, y):
    """O1 for any C (definite or not): (C^-1 y, log |det C|, sign det C) by dense LU with
    partial pivoting; y (n,) or (n, nrhs)."""
    x = _f64(x)
    n, d = (x.shape[0], 1) if x.ndim == 1 else x.shape
    Y, one = _cols(y)
    X = np.zeros_like(Y, order="F")
    ld, sg = ctypes.c_double(), ctypes.c_int()
    th = _theta(theta)
    _check(lib().oracle_dense_lu_solve(_d(x), n, d, KERNELS[kernel], _d(th), sigma2, _d(Y),
                                       Y.shape[1], n, _d(X), n, ctypes.byref(ld),
                                       ctypes.byref(sg)), "dense_lu_solve")
    return (X[:, 0] if one else X), ld.value, sg.value


def dense_matvec_rows(x, kernel, theta, sigma2, v, rows):
    """Exact (C v)[rows] in FP64 with compensated summation, O(n) per row."""
    x = _f64(x)
    n, d = (x.shape[0], 1) if x.ndim == 1 else x.shape
    v = _f64(v)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty(rows.size)
    th = _theta(theta)
    lib().oracle_dense_matvec_rows(_d(x), n, d, KERNELS[kernel], _d(th), sigma2, _d(v),
                                   rows.ctypes.data_as(_lp), rows.size, _d(out))
    return out


def ou_closed_form(xs_sorted, ell, amp, sigma2, y_sorted):
    """OU (exponential kernel) closed form on sorted 1-D points: (C^-1 y, log det C)."""
    xs = _f64(xs_sorted).reshape(-1)
    Y, one = _cols(y_sorted)
    X = np.zeros_like(Y, order="F")
    ld = ctypes.c_double()
    n = xs.size
    _check(lib().oracle_ou_closed_form(_d(xs), n, ell, amp, sigma2, _d(Y), Y.shape[1], n, _d(X), n,
                                       ctypes.byref(ld)), "ou_closed_form")
    return (X[:, 0] if one else X), ld.value


def matern_kalman(xs_sorted, nu2: int, ell, amp, sigma2, y_sorted):
    """Kalman filter for Matern nu = nu2/2 on sorted 1-D points: (log det C, y^T C^-1 y)."""
    xs = _f64(xs_sorted).reshape(-1)
    y = _f64(y_sorted).reshape(-1)
    ld = ctypes.c_double()
    q = ctypes.c_double()
    _check(lib().oracle_matern_kalman(_d(xs), xs.size, nu2, ell, amp, sigma2, _d(y),
                                      ctypes.byref(ld), ctypes.byref(q)), "matern_kalman")
    return ld.value, q.value


def lu_logdet(A):
    A = _f64(A)
    sg = ctypes.c_int()
    v = lib().oracle_lu_logdet(_d(A), A.shape[0], ctypes.byref(sg))
    return v, sg.value


def lu_solve(A, b):
    A = _f64(A)
    b = _f64(b)
    x = np.empty_like(b)
    lib().oracle_lu_solve_dense(_d(A), A.shape[0], _d(b), _d(x))
    return x


def kappa(n: int, leaf: int) -> int:
    return lib().oracle_kappa(n, leaf)


def tree_order(x, leaf: int) -> np.ndarray:
    x = _f64(x)
    n, d = (x.shape[0], 1) if x.ndim == 1 else x.shape
    perm = np.empty(n, dtype=np.int64)
    lib().oracle_tree_order(_d(x), n, d, leaf, perm.ctypes.data_as(_lp))
    return perm


class Hodlr:
    """O2: the plain CPU HODLR factorization (same call sequence as the C-ABI)."""

    def __init__(self, x, kernel, theta, sigma2, leaf, eps, max_rank=64, allow_rank_cap=False,
                 compression: str = "aca"):
        """compression: "aca" (adaptive cross approximation) or "chebyshev" (analytic
        interpolation, 1-D)."""
        x = _f64(x)
        self.n, self.d = (x.shape[0], 1) if x.ndim == 1 else x.shape
        st = ctypes.c_int()
        th = _theta(theta)
        self._h = lib().oracle_hodlr_build(_d(x), self.n, self.d, KERNELS[kernel], _d(th), sigma2,
                                           leaf, eps, max_rank,
                                           {"aca": 0, "chebyshev": 1}[compression],
                                           ctypes.byref(st))
        if not self._h:
            raise OracleError(f"build: status {STATUS.get(st.value, st.value)}")
        self.status = st.value
        if st.value != 0 and not allow_rank_cap:
            lib().oracle_hodlr_destroy(self._h)
            self._h = None
            raise OracleError(f"build: status {STATUS.get(st.value, st.value)}")
        self.kappa = lib().oracle_hodlr_kappa(self._h)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().oracle_hodlr_destroy(self._h)
            self._h = None

    def ranks(self) -> np.ndarray:
        m = (1 << self.kappa) - 1
        out = np.zeros(max(m, 1), dtype=np.int32)
        lib().oracle_hodlr_ranks(self._h, out.ctypes.data_as(_ip), m)
        return out[:m]

    def perm(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.int64)
        lib().oracle_hodlr_perm(self._h, out.ctypes.data_as(_lp))
        return out

    def factor(self):
        _check(lib().oracle_hodlr_factor(self._h), "factor")

    def factor_solve(self, y):
        Y, one = _cols(y)
        X = np.zeros_like(Y, order="F")
        _check(lib().oracle_hodlr_factor_solve(self._h, _d(Y), _d(X), Y.shape[1], self.n),
               "factor_solve")
        return X[:, 0] if one else X

    def solve(self, y):
        Y, one = _cols(y)
        X = np.zeros_like(Y, order="F")
        _check(lib().oracle_hodlr_solve(self._h, _d(Y), _d(X), Y.shape[1], self.n), "solve")
        return X[:, 0] if one else X

    def logdet(self) -> float:
        v = ctypes.c_double()
        _check(lib().oracle_hodlr_logdet(self._h, ctypes.byref(v)), "logdet")
        return v.value

    def logdet_sign(self) -> int:
        v = ctypes.c_int()
        _check(lib().oracle_hodlr_logdet_sign(self._h, ctypes.byref(v)), "logdet_sign")
        return v.value

    def level_logdets(self):
        nl = 1 << self.kappa
        leaf = np.empty(nl)
        node = np.empty(max(nl - 1, 1))
        lib().oracle_hodlr_level_logdets(self._h, _d(leaf), _d(node))
        return leaf, node[: nl - 1]

    def loglik(self, y) -> float:
        y = _f64(y).reshape(-1)
        v = ctypes.c_double()
        _check(lib().oracle_hodlr_loglik(self._h, _d(y), ctypes.byref(v)), "loglik")
        return v.value

    def matvec(self, v):
        v = _f64(v).reshape(-1)
        out = np.empty_like(v)
        lib().oracle_hodlr_matvec(self._h, _d(v), _d(out))
        return out

    def node_factors(self, node_id: int):
        b, s = ctypes.c_int64(), ctypes.c_int64()
        lib().oracle_hodlr_node_range(self._h, 2 * node_id + 1, ctypes.byref(b), ctypes.byref(s))
        ml = s.value
        lib().oracle_hodlr_node_range(self._h, 2 * node_id + 2, ctypes.byref(b), ctypes.byref(s))
        mr = s.value
        r = lib().oracle_hodlr_node_factors(self._h, node_id, None, None)
        U = np.zeros((r, ml))
        V = np.zeros((r, mr))
        lib().oracle_hodlr_node_factors(self._h, node_id, _d(U), _d(V))
        return U.T.copy(), V.T.copy()

    def node_range(self, node_id: int):
        b, s = ctypes.c_int64(), ctypes.c_int64()
        lib().oracle_hodlr_node_range(self._h, node_id, ctypes.byref(b), ctypes.byref(s))
        return b.value, s.value
