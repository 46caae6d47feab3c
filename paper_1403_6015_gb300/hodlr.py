"""Python binding of the C ABI in include/hodlr.h (argument marshalling only).

Every step of the computation runs in libhodlr_gb300.so's CUDA kernels. Arrays may be
numpy arrays (host; the library copies them) or torch CUDA tensors (device; stream
ordered). There is no CPU fallback: if the library is missing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhodlr_gb300.so")

KERNELS = {"exp": 0, "se": 1, "matern32": 2, "matern52": 3, "rq": 4, "imq": 5, "mq": 6,
           "biharmonic": 7}
INDEFINITE = ("mq", "biharmonic")  # LU leaves, signed log |det|, no log-likelihood
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ENOTSPD", 4: "ERANK", 5: "ETIMEOUT",
          6: "ESTATE", 7: "ECUDA"}
HODLR_OK, HODLR_EINVAL, HODLR_ENOMEM, HODLR_ENOTSPD, HODLR_ERANK = 0, 1, 2, 3, 4
HODLR_ETIMEOUT, HODLR_ESTATE, HODLR_ECUDA = 5, 6, 7


class hodlr_batch_lane(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("theta", ctypes.c_void_p), ("sigma2", ctypes.c_void_p),
                ("y", ctypes.c_void_p), ("out", ctypes.c_void_p), ("status", ctypes.c_void_p),
                ("first", ctypes.c_int64), ("stride", ctypes.c_int64), ("count", ctypes.c_int64)]


class hodlr_tuning(ctypes.Structure):
    _fields_ = [("leaf_threads", ctypes.c_int), ("sweep_mode", ctypes.c_int),
                ("leaf_kernel", ctypes.c_int), ("sweep_tile", ctypes.c_int)]


class hodlr_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("rank_mode", ctypes.c_int),
                ("max_rank", ctypes.c_int), ("max_nrhs", ctypes.c_int),
                ("refine_tol", ctypes.c_double), ("refine_maxit", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("rq_alpha", ctypes.c_double),
                ("compression", ctypes.c_int)]


_lib = None
_vp = ctypes.c_void_p
_dp = ctypes.c_void_p  # host or device double*, passed as an address


def load():
    """Load the CUDA library (build it first with build_lib.build()). Raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "paper_1403_6015_gb300.build_lib.build() (no CPU fallback exists)")
    L = ctypes.CDLL(LIB_PATH)
    L.hodlr_default_opts.argtypes = [ctypes.POINTER(hodlr_opts)]
    L.hodlr_build.argtypes = [_dp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double,
                              ctypes.c_int, ctypes.c_double, ctypes.POINTER(hodlr_opts),
                              ctypes.POINTER(_vp)]
    L.hodlr_rebuild.argtypes = [_vp, _dp, ctypes.c_double]
    L.hodlr_factor.argtypes = [_vp]
    L.hodlr_factor_solve.argtypes = [_vp, _dp, _dp, ctypes.c_int, ctypes.c_int64]
    L.hodlr_solve.argtypes = [_vp, _dp, _dp, ctypes.c_int, ctypes.c_int64]
    L.hodlr_logdet.argtypes = [_vp, _dp]
    L.hodlr_logdet_signed.argtypes = [_vp, _dp, ctypes.POINTER(ctypes.c_int)]
    L.hodlr_loglik.argtypes = [_vp, _dp, _dp]
    L.hodlr_ranks.argtypes = [_vp, _dp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
    L.hodlr_tree.argtypes = [_vp, ctypes.POINTER(ctypes.c_int), _dp]
    L.hodlr_matvec.argtypes = [_vp, _dp, _dp]
    L.hodlr_phase_ms.argtypes = [_vp, _dp]
    L.hodlr_counters.argtypes = [_vp, _dp]
    L.hodlr_refine_info.argtypes = [_vp, _dp, _dp]
    L.hodlr_predict.argtypes = [_vp, _dp, ctypes.c_int64, _dp, _dp, _dp]
    L.hodlr_get_tuning.argtypes = [_vp, ctypes.POINTER(hodlr_tuning)]
    L.hodlr_set_tuning.argtypes = [_vp, ctypes.POINTER(hodlr_tuning)]
    L.hodlr_autotune.argtypes = [_vp, _dp, ctypes.c_int, ctypes.POINTER(hodlr_tuning),
                                 ctypes.POINTER(ctypes.c_float)]
    L.hodlr_presize.argtypes = [_vp, _dp, ctypes.c_int]
    L.hodlr_status_flags.argtypes = [_vp, _dp]
    L.hodlr_loglik_sweep.argtypes = [_vp, ctypes.c_int64, _dp, _dp, _dp, _dp, _dp]
    L.hodlr_loglik_batched.argtypes = [ctypes.POINTER(hodlr_batch_lane), ctypes.c_int, _vp]
    L.hodlr_mlp_num_params.restype = ctypes.c_int
    L.hodlr_mlp_num_features.restype = ctypes.c_int
    L.hodlr_mlp_create.argtypes = [ctypes.c_uint64, _vp, ctypes.POINTER(_vp)]
    L.hodlr_mlp_destroy.argtypes = [_vp]
    L.hodlr_mlp_params.argtypes = [_vp, _dp, ctypes.c_int]
    L.hodlr_mlp_forward.argtypes = [_vp, _dp, ctypes.c_int64, _dp]
    L.hodlr_mlp_gradient.argtypes = [_vp, _dp, _dp, ctypes.c_int64, _dp, _dp]
    L.hodlr_mlp_train.argtypes = [_vp, _dp, _dp, ctypes.c_int64, ctypes.c_int, ctypes.c_float, _dp]
    L.hodlr_mlp_save.argtypes = [_vp, ctypes.c_char_p]
    L.hodlr_mlp_load.argtypes = [_vp, ctypes.c_char_p]
    L.hodlr_block_features.argtypes = [_vp, ctypes.c_double, _dp, ctypes.c_int64]
    L.hodlr_predict_ranks.argtypes = [_vp, _vp, ctypes.c_double, ctypes.c_int, _dp]
    L.hodlr_loglik_small_noalloc.argtypes = [_dp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _dp,
                                             ctypes.c_double, _dp, _dp, _vp]
    L.hodlr_last_error.argtypes = [_vp]
    L.hodlr_last_error.restype = ctypes.c_char_p
    L.hodlr_status_string.argtypes = [ctypes.c_int]
    L.hodlr_status_string.restype = ctypes.c_char_p
    L.hodlr_destroy.argtypes = [_vp]
    for name in ("hodlr_build", "hodlr_rebuild", "hodlr_factor", "hodlr_factor_solve",
                 "hodlr_solve", "hodlr_logdet", "hodlr_loglik", "hodlr_ranks", "hodlr_tree",
                 "hodlr_matvec", "hodlr_phase_ms", "hodlr_counters",
                 "hodlr_loglik_small_noalloc", "hodlr_presize", "hodlr_status_flags",
                 "hodlr_loglik_sweep", "hodlr_mlp_create", "hodlr_mlp_params",
                 "hodlr_mlp_forward", "hodlr_mlp_gradient", "hodlr_mlp_train", "hodlr_mlp_save",
                 "hodlr_mlp_load", "hodlr_block_features", "hodlr_predict_ranks",
                 "hodlr_loglik_batched", "hodlr_refine_info", "hodlr_get_tuning",
                 "hodlr_set_tuning", "hodlr_autotune", "hodlr_predict", "hodlr_logdet_signed"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


class HodlrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _addr(a) -> int:
    """Address of a numpy array or torch tensor's data."""
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _is_torch(a) -> bool:
    return hasattr(a, "data_ptr") and hasattr(a, "is_cuda")


def _f64_host(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---- the C ABI, name for name ------------------------------------------------------------

def hodlr_default_opts() -> hodlr_opts:
    o = hodlr_opts()
    load().hodlr_default_opts(ctypes.byref(o))
    return o


def hodlr_build(x, n, d, kernel, theta, sigma2, leaf, eps, opts=None):
    """Returns (status, ctx). x: host numpy (n, d) float64 or a CUDA tensor (row-major)."""
    L = load()
    th = _f64_host(theta)
    out = _vp()
    st = L.hodlr_build(_addr(x), n, d, kernel, th.ctypes.data, sigma2, leaf, eps,
                       ctypes.byref(opts) if opts is not None else None, ctypes.byref(out))
    return st, out.value


def hodlr_rebuild(ctx, theta, sigma2):
    th = _f64_host(theta)
    return load().hodlr_rebuild(ctx, th.ctypes.data, sigma2)


def hodlr_factor(ctx):
    return load().hodlr_factor(ctx)


def hodlr_factor_solve(ctx, y_addr, x_addr, nrhs, ld):
    return load().hodlr_factor_solve(ctx, y_addr, x_addr, nrhs, ld)


def hodlr_solve(ctx, y_addr, x_addr, nrhs, ld):
    return load().hodlr_solve(ctx, y_addr, x_addr, nrhs, ld)


def hodlr_logdet(ctx, out_addr):
    return load().hodlr_logdet(ctx, out_addr)


def hodlr_logdet_signed(ctx, out_addr, sign: "ctypes.c_int"):
    """log |det C| into out_addr (host or device), its sign into the ctypes int `sign`."""
    return load().hodlr_logdet_signed(ctx, out_addr, ctypes.byref(sign))


def hodlr_loglik(ctx, y_addr, out_addr):
    return load().hodlr_loglik(ctx, y_addr, out_addr)


def hodlr_ranks(ctx, buf, cap):
    cnt = ctypes.c_int64()
    st = load().hodlr_ranks(ctx, _addr(buf) if buf is not None else None, cap, ctypes.byref(cnt))
    return st, cnt.value


def hodlr_tree(ctx, perm=None):
    k = ctypes.c_int()
    st = load().hodlr_tree(ctx, ctypes.byref(k), _addr(perm) if perm is not None else None)
    return st, k.value


def hodlr_matvec(ctx, x_addr, y_addr):
    return load().hodlr_matvec(ctx, x_addr, y_addr)


def hodlr_phase_ms(ctx, buf):
    return load().hodlr_phase_ms(ctx, _addr(buf))


def hodlr_counters(ctx, buf):
    return load().hodlr_counters(ctx, _addr(buf))


def hodlr_get_tuning(ctx, out: hodlr_tuning):
    return load().hodlr_get_tuning(ctx, ctypes.byref(out))


def hodlr_set_tuning(ctx, t: hodlr_tuning):
    return load().hodlr_set_tuning(ctx, ctypes.byref(t))


def hodlr_autotune(ctx, y_addr, reps, best: hodlr_tuning, best_ms):
    """best_ms: a ctypes.c_float (or None)."""
    return load().hodlr_autotune(ctx, y_addr, reps, ctypes.byref(best),
                                 ctypes.byref(best_ms) if best_ms is not None else None)


def hodlr_predict(ctx, xtest_addr, m, y_addr, mean_addr, var_addr):
    return load().hodlr_predict(ctx, xtest_addr, m, y_addr, mean_addr, var_addr)


def hodlr_refine_info(ctx, corrections, residual):
    """corrections: int32 numpy array (1); residual: float64 numpy array (1)."""
    return load().hodlr_refine_info(ctx, _addr(corrections), _addr(residual))


def hodlr_loglik_small_noalloc(x_addr, n, d, kernel, theta, sigma2, y_addr, out_addr,
                               stream=None):
    """Device pointers only; n <= 128; no device allocation (see include/hodlr.h)."""
    th = _f64_host(theta)
    return load().hodlr_loglik_small_noalloc(x_addr, n, d, kernel, th.ctypes.data, sigma2,
                                             y_addr, out_addr, stream)


def hodlr_presize(ctx, level_ranks):
    """level_ranks: host int32 array of kappa entries, or None for adaptive mode."""
    if level_ranks is None:
        return load().hodlr_presize(ctx, None, 0)
    r = np.ascontiguousarray(level_ranks, dtype=np.int32)
    return load().hodlr_presize(ctx, r.ctypes.data, r.size)


def hodlr_status_flags(ctx):
    f = np.zeros(1, dtype=np.int32)
    st = load().hodlr_status_flags(ctx, f.ctypes.data)
    return st, int(f[0])


def hodlr_loglik_sweep(ctx, nset, theta_addr, sigma2_addr, y_addr, out_addr, status_addr=None):
    return load().hodlr_loglik_sweep(ctx, nset, theta_addr, sigma2_addr, y_addr, out_addr,
                                     status_addr)


def hodlr_loglik_batched(lanes, stream):
    """lanes: sequence of hodlr_batch_lane; stream: cudaStream_t handle (int)."""
    arr = (hodlr_batch_lane * len(lanes))(*lanes)
    return load().hodlr_loglik_batched(arr, len(lanes), stream)


def loglik_batched(contexts, theta, sigma2, y, out, status=None, stream=None):
    """Settings b of (theta (nset, 2), sigma2 (nset,)) on len(contexts) presized contexts of
    the same points, lane i taking settings i, i + L, ...; CUDA tensors throughout."""
    import torch
    nset = theta.shape[0]
    L = len(contexts)
    lanes = [hodlr_batch_lane(h._ctx, theta.data_ptr(), sigma2.data_ptr(), y.data_ptr(),
                              out.data_ptr(), status.data_ptr() if status is not None else None,
                              i, L, (nset - i + L - 1) // L)
             for i, h in enumerate(contexts) if i < nset]
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    st = hodlr_loglik_batched(lanes, s)
    if st != HODLR_OK:
        msgs = {hodlr_last_error(h._ctx) for h in contexts} - {""}
        raise HodlrError(st, "hodlr_loglik_batched: " + "; ".join(sorted(msgs)))
    return out


def hodlr_mlp_num_params() -> int:
    return load().hodlr_mlp_num_params()


def hodlr_mlp_num_features() -> int:
    return load().hodlr_mlp_num_features()


def hodlr_mlp_create(seed=0, stream=None):
    out = _vp()
    st = load().hodlr_mlp_create(seed, stream, ctypes.byref(out))
    return st, out.value


def hodlr_mlp_destroy(m):
    load().hodlr_mlp_destroy(m)


def hodlr_mlp_params(m, buf, set_):
    return load().hodlr_mlp_params(m, _addr(buf), 1 if set_ else 0)


def hodlr_mlp_forward(m, x_addr, n, y_addr):
    return load().hodlr_mlp_forward(m, x_addr, n, y_addr)


def hodlr_mlp_gradient(m, x_addr, t_addr, n, grad_addr, loss_addr):
    return load().hodlr_mlp_gradient(m, x_addr, t_addr, n, grad_addr, loss_addr)


def hodlr_mlp_train(m, x_addr, t_addr, n, steps, lr, loss_addr):
    return load().hodlr_mlp_train(m, x_addr, t_addr, n, steps, lr, loss_addr)


def hodlr_mlp_save(m, path):
    return load().hodlr_mlp_save(m, path.encode())


def hodlr_mlp_load(m, path):
    return load().hodlr_mlp_load(m, path.encode())


def hodlr_block_features(ctx, ell, x_addr, ld):
    return load().hodlr_block_features(ctx, ell, x_addr, ld)


def hodlr_predict_ranks(ctx, mlp, ell, margin, out):
    return load().hodlr_predict_ranks(ctx, mlp, ell, margin, _addr(out))


def hodlr_last_error(ctx) -> str:
    return load().hodlr_last_error(ctx).decode()


def hodlr_status_string(st: int) -> str:
    return load().hodlr_status_string(st).decode()


def hodlr_destroy(ctx):
    load().hodlr_destroy(ctx)


# ---- convenience object ------------------------------------------------------------------

class Hodlr:
    """One HODLR problem: C = sigma2 I + K(x; theta) on one GPU.

    x, y may be numpy arrays (host) or torch CUDA tensors (device). Outputs follow the
    input's kind: numpy in, numpy out; CUDA tensor in, CUDA tensor out.
    """

    def __init__(self, x, kernel: str, theta, sigma2: float, leaf: int, eps: float,
                 max_rank: int = 64, max_nrhs: int = 16, stream=None, allow_rank_cap=False,
                 precision: int = 0, refine_maxit: int = 0, refine_tol: float = 1e-10,
                 rq_alpha: float = 1.0, compression: str = "aca"):
        if _is_torch(x):
            if x.dtype.itemsize != 8 or not x.is_contiguous():
                raise ValueError("x must be a contiguous float64 tensor")
            self.n = x.shape[0]
            self.d = 1 if x.dim() == 1 else x.shape[1]
            xin = x
        else:
            xin = _f64_host(x)
            self.n = xin.shape[0]
            self.d = 1 if xin.ndim == 1 else xin.shape[1]
        o = hodlr_default_opts()
        o.max_rank = max_rank
        o.max_nrhs = max_nrhs
        o.precision = precision
        o.refine_maxit = refine_maxit
        o.refine_tol = refine_tol
        o.rq_alpha = rq_alpha
        o.compression = {"aca": 0, "chebyshev": 1}[compression]
        if stream is not None:
            o.stream = stream
        self.kernel = kernel
        self.precision = precision
        self.max_rank = max_rank
        st, ctx = hodlr_build(xin, self.n, self.d, KERNELS[kernel], theta, sigma2, leaf, eps, o)
        self.status = st
        if not ctx:
            raise HodlrError(st, "hodlr_build failed")
        self._ctx = ctx
        if st not in (HODLR_OK,) and not (st == HODLR_ERANK and allow_rank_cap):
            msg = hodlr_last_error(ctx)
            self.close()
            raise HodlrError(st, msg)

    def close(self):
        if getattr(self, "_ctx", None):
            hodlr_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != HODLR_OK:
            raise HodlrError(st, f"{what}: {hodlr_last_error(self._ctx)}")

    def rebuild(self, theta, sigma2):
        self._check(hodlr_rebuild(self._ctx, theta, sigma2), "rebuild")

    def factor(self):
        self._check(hodlr_factor(self._ctx), "factor")

    @staticmethod
    def _cols(y):
        if _is_torch(y):
            one = y.dim() == 1
            Y = y.reshape(-1, 1) if one else y
            # column-major: a (nrhs, n) contiguous tensor viewed transposed
            Yc = Y.t().contiguous() if not one else Y.contiguous()
            return Yc, one, True
        y = np.asarray(y, dtype=np.float64)
        one = y.ndim == 1
        Y = np.asfortranarray(y.reshape(-1, 1) if one else y)
        return Y, one, False

    def _out_like(self, Y, is_t):
        if is_t:
            import torch
            return torch.empty_like(Y)
        return np.zeros_like(Y, order="F")

    @staticmethod
    def _result(X, one, is_t):
        if is_t:
            return X.reshape(-1) if one else X.t()
        return X[:, 0] if one else X

    def factor_solve(self, y):
        Y, one, is_t = self._cols(y)
        X = self._out_like(Y, is_t)
        nrhs = 1 if one else (Y.shape[0] if is_t else Y.shape[1])
        self._check(hodlr_factor_solve(self._ctx, _addr(Y), _addr(X), nrhs, self.n), "factor_solve")
        return self._result(X, one, is_t)

    def solve(self, y):
        Y, one, is_t = self._cols(y)
        X = self._out_like(Y, is_t)
        nrhs = 1 if one else (Y.shape[0] if is_t else Y.shape[1])
        self._check(hodlr_solve(self._ctx, _addr(Y), _addr(X), nrhs, self.n), "solve")
        return self._result(X, one, is_t)

    def logdet(self, out=None) -> float:
        buf = out if out is not None else np.zeros(1)
        self._check(hodlr_logdet(self._ctx, _addr(buf)), "logdet")
        return buf if out is not None else float(buf[0])

    def logdet_signed(self):
        """(log |det C|, sign of det C); the sign is -1 only for an indefinite kernel."""
        buf = np.zeros(1)
        sg = ctypes.c_int()
        self._check(hodlr_logdet_signed(self._ctx, _addr(buf), sg), "logdet_signed")
        return float(buf[0]), sg.value

    def loglik(self, y, out=None):
        if _is_torch(y):
            yy = y.contiguous()
        else:
            yy = _f64_host(y).reshape(-1)
        buf = out if out is not None else np.zeros(1)
        self._check(hodlr_loglik(self._ctx, _addr(yy), _addr(buf)), "loglik")
        return buf if out is not None else float(buf[0])

    def ranks(self) -> np.ndarray:
        st, cnt = hodlr_ranks(self._ctx, None, 0)
        buf = np.zeros(max(cnt, 1), dtype=np.int32)
        self._check(hodlr_ranks(self._ctx, buf, cnt)[0], "ranks")
        return buf[:cnt]

    def tree(self):
        perm = np.zeros(self.n, dtype=np.int64)
        st, kappa = hodlr_tree(self._ctx, perm)
        self._check(st, "tree")
        return kappa, perm

    def matvec(self, x):
        if _is_torch(x):
            xx = x.contiguous()
            import torch
            out = torch.empty_like(xx)
        else:
            xx = _f64_host(x).reshape(-1)
            out = np.zeros_like(xx)
        self._check(hodlr_matvec(self._ctx, _addr(xx), _addr(out)), "matvec")
        return out

    def phase_ms(self):
        buf = np.zeros(6, dtype=np.float32)
        self._check(hodlr_phase_ms(self._ctx, buf), "phase_ms")
        return {"ordering": float(buf[0]), "compression": float(buf[1]),
                "factor": float(buf[2]), "solve": float(buf[3]),
                "leaf_kernel": float(buf[4]), "levels": float(buf[5])}

    def level_ranks(self) -> np.ndarray:
        """Largest rank of each level from the last adaptive compression."""
        r = self.ranks()
        kappa = self.tree()[0]
        return np.array([int(r[(1 << j) - 1:(1 << (j + 1)) - 1].max()) for j in range(kappa)],
                        dtype=np.int32)

    def presize(self, level_ranks):
        self._check(hodlr_presize(self._ctx, level_ranks), "presize")

    def status_flags(self) -> int:
        st, f = hodlr_status_flags(self._ctx)
        self._check(st, "status_flags")
        return f

    def loglik_sweep(self, theta, sigma2, y, out=None, status=None):
        """theta: CUDA tensor (nset, 2); sigma2, y: CUDA tensors; returns out (nset,)."""
        import torch
        nset = theta.shape[0]
        if out is None:
            out = torch.empty(nset, dtype=torch.float64, device=theta.device)
        self._check(hodlr_loglik_sweep(self._ctx, nset, theta.data_ptr(), sigma2.data_ptr(),
                                       y.data_ptr(), out.data_ptr(),
                                       status.data_ptr() if status is not None else None),
                    "loglik_sweep")
        return out

    def block_features(self, ell):
        """Features of every off-diagonal block (torch CUDA tensor, (2^kappa - 1) x 12)."""
        import torch
        m = (1 << self.tree()[0]) - 1
        X = torch.empty((max(m, 1), 12), dtype=torch.float32, device="cuda")
        self._check(hodlr_block_features(self._ctx, ell, X.data_ptr(), 12), "block_features")
        return X[:m]

    def predict_level_ranks(self, mlp, ell, margin=1):
        out = np.zeros(max(self.tree()[0], 1), dtype=np.int32)
        self._check(hodlr_predict_ranks(self._ctx, mlp._m, ell, margin, out), "predict_ranks")
        return out[:self.tree()[0]]

    def counters(self):
        buf = np.zeros(2, dtype=np.int64)
        self._check(hodlr_counters(self._ctx, buf), "counters")
        return {"launches": int(buf[0]), "syncs": int(buf[1])}

    def tuning(self) -> dict:
        t = hodlr_tuning()
        self._check(hodlr_get_tuning(self._ctx, t), "get_tuning")
        return {"leaf_threads": t.leaf_threads, "sweep_mode": t.sweep_mode,
                "leaf_kernel": t.leaf_kernel, "sweep_tile": t.sweep_tile}

    def set_tuning(self, leaf_threads: int, sweep_mode: int = 0, leaf_kernel: int | None = None,
                   sweep_tile: int | None = None):
        cur = self.tuning()
        if leaf_kernel is None:
            leaf_kernel = cur["leaf_kernel"]
        if sweep_tile is None:
            sweep_tile = cur["sweep_tile"]
        t = hodlr_tuning(leaf_threads, sweep_mode, leaf_kernel, sweep_tile)
        self._check(hodlr_set_tuning(self._ctx, t), "set_tuning")

    def autotune(self, y, reps: int = 3, cache: str | None = None) -> dict:
        """Time the launch configurations on this problem and keep the fastest. With a
        cache file (JSON), a configuration stored for the same GPU and problem shape is
        applied without timing, and new results are added to it."""
        import json
        key = None
        if cache is not None:
            import torch
            kappa = self.tree()[0]
            r = self.ranks()
            lv = [int(r[(1 << j) - 1:(1 << (j + 1)) - 1].max()) for j in range(kappa)] if r.size else []
            key = "|".join(str(v) for v in (torch.cuda.get_device_name(), self.n, self.d, self.kernel,
                                            self.precision, kappa, tuple(lv)))
            try:
                with open(cache) as f:
                    table = json.load(f)
            except (OSError, ValueError):
                table = {}
            if key in table:
                self.set_tuning(table[key]["leaf_threads"], table[key]["sweep_mode"],
                                table[key].get("leaf_kernel", 0), table[key].get("sweep_tile", 0))
                return dict(table[key], cached=True)
        yy = y.contiguous() if _is_torch(y) else _f64_host(y).reshape(-1)
        best = hodlr_tuning()
        ms = ctypes.c_float()
        self._check(hodlr_autotune(self._ctx, _addr(yy), reps, best, ms), "autotune")
        res = {"leaf_threads": best.leaf_threads, "sweep_mode": best.sweep_mode,
               "leaf_kernel": best.leaf_kernel, "sweep_tile": best.sweep_tile, "ms": ms.value}
        if key is not None:
            table[key] = res
            with open(cache, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
        return dict(res, cached=False)

    def predict(self, xtest, y, var: bool = True):
        """Posterior mean (and latent variance) at the test points with the current
        factorization. numpy in, numpy out; CUDA tensors in, CUDA tensors out."""
        if _is_torch(xtest):
            import torch
            xt = xtest.contiguous()
            m = xt.shape[0]
            yy = y.contiguous()
            mean = torch.empty(m, dtype=torch.float64, device=xt.device)
            vv = torch.empty(m, dtype=torch.float64, device=xt.device) if var else None
        else:
            xt = _f64_host(xtest).reshape(len(xtest), -1)
            m = xt.shape[0]
            yy = _f64_host(y).reshape(-1)
            mean = np.zeros(m)
            vv = np.zeros(m) if var else None
        self._check(hodlr_predict(self._ctx, _addr(xt), m, _addr(yy), _addr(mean),
                                  _addr(vv) if vv is not None else None), "predict")
        return (mean, vv) if var else mean

    def refine_info(self):
        """(corrections, final relative residual) of the last solve's refinement."""
        k = np.zeros(1, dtype=np.int32)
        r = np.zeros(1, dtype=np.float64)
        self._check(hodlr_refine_info(self._ctx, k, r), "refine_info")
        return int(k[0]), float(r[0])
