"""Learned rank predictor: the network object, pair collection and training.

The network (12 -> 64 -> 64 -> 1, tanh) and its training run in libhodlr_gb300.so
(hodlr_mlp_*); this module only gathers (block features, rank) pairs from the FP64
compressor over a grid of problems and calls the library.
"""
from __future__ import annotations

import numpy as np

from . import hodlr as H


class RankMLP:
    def __init__(self, seed: int = 0, stream=None):
        st, m = H.hodlr_mlp_create(seed, stream)
        if st != H.HODLR_OK:
            raise H.HodlrError(st, "hodlr_mlp_create")
        self._m = m

    def close(self):
        if getattr(self, "_m", None):
            H.hodlr_mlp_destroy(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        p = np.zeros(H.hodlr_mlp_num_params(), dtype=np.float32)
        H.hodlr_mlp_params(self._m, p, False)
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        H.hodlr_mlp_params(self._m, p, True)

    def forward(self, X):
        import torch
        Y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        st = H.hodlr_mlp_forward(self._m, X.data_ptr(), X.shape[0], Y.data_ptr())
        if st != H.HODLR_OK:
            raise H.HodlrError(st, "hodlr_mlp_forward")
        torch.cuda.synchronize()
        return Y

    def gradient(self, X, T):
        g = np.zeros(H.hodlr_mlp_num_params(), dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        st = H.hodlr_mlp_gradient(self._m, X.data_ptr(), T.data_ptr(), X.shape[0], g.ctypes.data,
                                  loss.ctypes.data)
        if st != H.HODLR_OK:
            raise H.HodlrError(st, "hodlr_mlp_gradient")
        return g, float(loss[0])

    def train(self, X, T, steps: int, lr: float = 1e-3) -> float:
        loss = np.zeros(1, dtype=np.float32)
        st = H.hodlr_mlp_train(self._m, X.data_ptr(), T.data_ptr(), X.shape[0], steps, lr,
                               loss.ctypes.data)
        if st != H.HODLR_OK:
            raise H.HodlrError(st, "hodlr_mlp_train")
        return float(loss[0])

    def save(self, path: str):
        if H.hodlr_mlp_save(self._m, path) != H.HODLR_OK:
            raise IOError(path)

    def load(self, path: str):
        if H.hodlr_mlp_load(self._m, path) != H.HODLR_OK:
            raise IOError(path)


def collect_pairs(problems, max_rank: int = 64):
    """(features, log(1 + rank)) of every block of every problem, from the FP64 compressor.

    problems: iterable of (x, kernel, ell, sigma2, leaf, eps). Returns torch CUDA tensors
    X (N x 12, float32) and T (N, float32), and the raw ranks (numpy).
    """
    import torch
    Xs, Ts, R = [], [], []
    for x, kern, ell, s2, leaf, eps in problems:
        h = H.Hodlr(x, kern, [ell, 1.0], s2, leaf, eps, max_rank=max_rank, allow_rank_cap=True)
        r = h.ranks()
        if r.size == 0:
            continue
        Xs.append(h.block_features(ell).clone())
        Ts.append(torch.from_numpy(np.log1p(r.astype(np.float32))).cuda())
        R.append(r)
        h.close()
    return torch.cat(Xs), torch.cat(Ts), np.concatenate(R)


def presize_profile(h, net, ell: float, margin: int = 1, scale: float = 1.0):
    """Per-level presize from the network: ceil(scale x predicted rank) + margin, capped at
    the context's max_rank - 1 (the regression is on log(1 + r), so its errors are
    relative: scale > 1 covers them at high ranks, margin at low ones)."""
    p0 = h.predict_level_ranks(net, float(ell), 0).astype(np.float64)
    pre = np.ceil(p0 * scale).astype(np.int32) + margin
    return np.minimum(pre, h.max_rank - 1).astype(np.int32)


def run_presized(h, ells, sigma2s, y, groups, lanes=None, stream=None):
    """Evaluate settings group by group, each group presized to its level profile: a
    captured graph on h replayed per setting, or, with lanes (contexts of the same points,
    each on its own stream, not stream), batched rounds over the lanes
    (hodlr_loglik_batched). Settings whose evaluation flagged a block above its presize
    are re-evaluated by the adaptive path (the fallback). groups: list of (indices,
    profile). Returns (loglik array, number of fallbacks)."""
    import torch
    ells = np.asarray(ells, dtype=np.float64)
    sigma2s = np.asarray(sigma2s, dtype=np.float64)
    out = np.zeros(len(ells))
    fallback = []
    for idx, prof in groups:
        prof = np.asarray(prof, dtype=np.int32)
        theta = torch.from_numpy(np.stack([ells[idx], np.ones(len(idx))], 1).copy()).cuda()
        sig = torch.from_numpy(sigma2s[idx].copy()).cuda()
        status = torch.zeros(len(idx), dtype=torch.int32, device="cuda")
        if lanes:
            for c in lanes:
                c.presize(prof)
            res = torch.zeros(len(idx), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            H.loglik_batched(lanes, theta, sig, y, res, status, stream=stream)
        else:
            h.presize(prof)
            res = h.loglik_sweep(theta, sig, y, status=status)
        torch.cuda.synchronize()
        out[idx] = res.cpu().numpy()
        fallback.extend(np.asarray(idx)[status.cpu().numpy() != 0].tolist())
    h.presize(None)
    for b in fallback:
        h.rebuild([float(ells[b]), 1.0], float(sigma2s[b]))
        out[b] = h.loglik(y)
    return out, len(fallback)


def sweep_with_predictor(h, net, ells, sigma2s, y, margin: int = 1, max_groups: int = 4,
                         scale: float = 1.0, lanes=None, stream=None):
    """Log-likelihoods of the settings (ells[b], sigma2s[b]) on the context h, presized by
    the network's predicted per-level ranks (presize_profile), with the adaptive path as the
    fallback for every setting whose evaluation flagged a rank above its presize.

    Settings are sorted by predicted total rank and cut into at most max_groups chunks of
    equal count; a chunk is presized to the elementwise maximum of its members' profiles
    and run by run_presized. y: CUDA tensor. Returns (loglik array, stats)."""
    ells = np.asarray(ells, dtype=np.float64)
    profs = np.array([presize_profile(h, net, e, margin, scale) for e in ells], dtype=np.int32)
    order = np.argsort(profs.sum(axis=1), kind="stable")
    chunks = [c for c in np.array_split(order, min(max_groups, len(ells))) if len(c)]
    groups = [(idx, profs[idx].max(axis=0)) for idx in chunks]
    out, nfb = run_presized(h, ells, sigma2s, y, groups, lanes=lanes, stream=stream)
    return out, {"groups": len(chunks), "fallbacks": nfb,
                 "distinct_profiles": len({tuple(p) for p in profs}),
                 "presized_rank_sum": int(sum(len(idx) * int(np.sum(pr)) for idx, pr in groups))}


def sweep_with_probe(h, ells, sigma2s, y, margin: int = 1, lanes=None, stream=None):
    """The same sweep without the network, the baseline of equal batching: one adaptive
    compression at the sweep's smallest length scale (where these covariances' blocks have
    their largest ranks) gives every level's rank, all settings run presized to it plus
    margin in one group (run_presized, the same lanes), and a setting that needs more falls
    back to the adaptive path. Returns (loglik array, stats)."""
    ells = np.asarray(ells, dtype=np.float64)
    sigma2s = np.asarray(sigma2s, dtype=np.float64)
    i0 = int(np.argmin(ells))
    h.presize(None)
    h.rebuild([float(ells[i0]), 1.0], float(sigma2s[i0]))
    prof = np.minimum(h.level_ranks() + margin, h.max_rank - 1).astype(np.int32)
    out, nfb = run_presized(h, ells, sigma2s, y, [(np.arange(len(ells)), prof)], lanes=lanes,
                            stream=stream)
    return out, {"groups": 1, "fallbacks": nfb, "probe_level_ranks": prof.tolist(),
                 "presized_rank_sum": int(len(ells) * int(np.sum(prof)))}


def _lane_buffers(ells, sigma2s, y):
    import torch
    theta = torch.from_numpy(np.stack([ells, np.ones(len(ells))], 1).copy()).cuda()
    sig = torch.from_numpy(np.asarray(sigma2s, dtype=np.float64).copy()).cuda()
    out = torch.zeros(len(ells), dtype=torch.float64, device="cuda")
    status = torch.full((len(ells),), -1, dtype=torch.int32, device="cuda")
    return theta, sig, y, out, status


def instances_presized(ctxs, settings, ys, profiles, stream):
    """Independent problems (contexts ctxs, each on its own stream), each presized to its
    profile and evaluated at its settings (ells, sigma2s) by one batched launch over all of
    them (hodlr_loglik_batched); settings that flagged a block above its presize fall back
    to the adaptive path. Returns (list of loglik arrays, fallbacks)."""
    import torch
    lanes, keep = [], []
    for h, (e, s2), y, prof in zip(ctxs, settings, ys, profiles):
        h.presize(np.asarray(prof, dtype=np.int32))
        theta, sig, yd, out, status = _lane_buffers(np.asarray(e, dtype=np.float64), s2, y)
        lanes.append(H.hodlr_batch_lane(h._ctx, theta.data_ptr(), sig.data_ptr(), yd.data_ptr(),
                                        out.data_ptr(), status.data_ptr(), 0, 1, len(e)))
        keep.append((theta, sig, out, status))
    torch.cuda.synchronize()
    st = H.hodlr_loglik_batched(lanes, stream)
    if st != H.HODLR_OK:
        raise H.HodlrError(st, "hodlr_loglik_batched")
    torch.cuda.synchronize()
    res, nfb = [], 0
    for h, (e, s2), y, (theta, sig, out, status) in zip(ctxs, settings, ys, keep):
        v = out.cpu().numpy()
        bad = np.nonzero(status.cpu().numpy() != 0)[0]
        if len(bad):
            h.presize(None)
            for b in bad:
                h.rebuild([float(e[b]), 1.0], float(s2[b]))
                v[b] = h.loglik(y)
            nfb += len(bad)
        res.append(v)
    return res, nfb


def instances_with_probe(ctxs, settings, ys, stream, margin: int = 0):
    """Baseline without the network: each problem's profile comes from one adaptive
    compression at its smallest length scale (an adaptive evaluation per problem, with its
    host synchronisations), then instances_presized."""
    profs = []
    for h, (e, s2) in zip(ctxs, settings):
        i0 = int(np.argmin(e))
        h.presize(None)
        h.rebuild([float(e[i0]), 1.0], float(s2[i0]))
        profs.append(np.minimum(h.level_ranks() + margin, h.max_rank - 1))
    res, nfb = instances_presized(ctxs, settings, ys, profs, stream)
    return res, {"fallbacks": nfb, "presized_rank_sum": int(sum(int(np.sum(p)) for p in profs))}


def instances_with_predictor(ctxs, net, settings, ys, stream, margin: int = 1, scale: float = 1.0):
    """The network presizes each problem (elementwise maximum of its settings' predicted
    profiles; no adaptive compression), then instances_presized."""
    profs = []
    for h, (e, s2) in zip(ctxs, settings):
        p = np.max([presize_profile(h, net, float(v), margin, scale) for v in e], axis=0)
        profs.append(p.astype(np.int32))
    res, nfb = instances_presized(ctxs, settings, ys, profs, stream)
    return res, {"fallbacks": nfb, "presized_rank_sum": int(sum(int(np.sum(p)) for p in profs))}
