"""Batched evaluation: one CUDA graph forks a round of evaluations into several presized
contexts (lanes) on their own streams; every result must equal the adaptive single
evaluation of the same setting and, for the Matern covariances in 1-D, the exact
log-likelihood of the oracle's Kalman filter (the state-space form cited in Sec. 2.3)."""
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


def kalman_loglik(x, y, nu2, ell, s2):
    """Exact Gaussian log-likelihood of Matern nu = nu2/2 (amplitude 1) on 1-D points."""
    order = np.argsort(x[:, 0], kind="stable")
    ld, q = O.matern_kalman(x[order, 0], nu2, ell, 1.0, s2, y[order])
    return -0.5 * q - 0.5 * ld - 0.5 * len(y) * np.log(2.0 * np.pi)


def settings(nset, seed):
    u = I.uniform01(seed, 2 * nset)
    ell = np.exp(np.log(0.05) + u[:nset] * (np.log(2.0) - np.log(0.05)))
    s2 = np.exp(np.log(1e-4) + u[nset:] * (np.log(1.0) - np.log(1e-4)))
    return ell, s2


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_sweep_lanes(H, precision):
    import torch
    n, nset, L = 1 << 14, 32, 8
    x, y = I.workload_1d(n, 1010)
    ell, s2 = settings(nset, 81)
    streams = [torch.cuda.Stream() for _ in range(L)]
    ctxs = []
    for s in streams:
        h = H.Hodlr(x, "matern52", [ell[0], 1.0], s2[0], 128, 1e-12, precision=precision,
                    stream=s.cuda_stream)
        h.presize(np.full(h.tree()[0], 4, dtype=np.int32))
        ctxs.append(h)
    theta = torch.from_numpy(np.stack([ell, np.ones(nset)], 1).copy()).cuda()
    sig = torch.from_numpy(s2.copy()).cuda()
    yd = torch.from_numpy(y).cuda()
    out = torch.zeros(nset, dtype=torch.float64, device="cuda")
    status = torch.full((nset,), -1, dtype=torch.int32, device="cuda")
    origin = torch.cuda.Stream()
    torch.cuda.synchronize()
    H.loglik_batched(ctxs, theta, sig, yd, out, status, stream=origin.cuda_stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert (status.cpu().numpy() == 0).all()
    for b in range(nset):
        r = H.Hodlr(x, "matern52", [ell[b], 1.0], s2[b], 128, 1e-12, precision=precision).loglik(y)
        assert abs(got[b] - r) <= 1e-12 * abs(r), (b, got[b], r)
        k = kalman_loglik(x, y, 5, ell[b], s2[b])
        assert abs(got[b] - k) <= 1e-9 * abs(k), (b, ell[b], s2[b], got[b], k)


def test_batched_uneven_instances(H):
    """Independent problems of uneven size (n log-uniform in [2^12, 2^15]), one lane each,
    three settings per problem."""
    import torch
    rng_n = I.uniform01(555, 6)
    sizes = np.round(np.exp(np.log(4096) + rng_n * (np.log(32768) - np.log(4096)))).astype(int)
    nset = 3
    lanes, keep = [], []
    origin = torch.cuda.Stream()
    for i, n in enumerate(sizes):
        x, y = I.workload_1d(int(n), 1100 + i)
        ell, s2 = settings(nset, 200 + i)
        s = torch.cuda.Stream()
        h = H.Hodlr(x, "matern32", [ell[0], 1.0], s2[0], 64, 1e-12, stream=s.cuda_stream)
        h.presize(np.full(h.tree()[0], 3, dtype=np.int32))
        theta = torch.from_numpy(np.stack([ell, np.ones(nset)], 1).copy()).cuda()
        sig = torch.from_numpy(s2.copy()).cuda()
        yd = torch.from_numpy(y).cuda()
        out = torch.zeros(nset, dtype=torch.float64, device="cuda")
        st = torch.full((nset,), -1, dtype=torch.int32, device="cuda")
        lanes.append(H.hodlr_batch_lane(h._ctx, theta.data_ptr(), sig.data_ptr(), yd.data_ptr(),
                                        out.data_ptr(), st.data_ptr(), 0, 1, nset))
        keep.append((h, s, x, y, ell, s2, theta, sig, yd, out, st))
    torch.cuda.synchronize()
    assert H.hodlr_loglik_batched(lanes, origin.cuda_stream) == H.HODLR_OK
    torch.cuda.synchronize()
    for h, s, x, y, ell, s2, theta, sig, yd, out, st in keep:
        assert (st.cpu().numpy() == 0).all()
        got = out.cpu().numpy()
        for b in range(nset):
            r = H.Hodlr(x, "matern32", [ell[b], 1.0], s2[b], 64, 1e-12).loglik(y)
            assert abs(got[b] - r) <= 1e-12 * abs(r)
            k = kalman_loglik(x, y, 3, ell[b], s2[b])
            assert abs(got[b] - k) <= 1e-9 * abs(k), (b, ell[b], s2[b], got[b], k)


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_uneven_matern52_instances_vs_kalman(H, precision):
    """The uneven-instance workload as the bench runs it: 64 independent problems with n
    log-uniform in [2^12, 2^18], Matern-5/2 (exact rank 3), leaf 128, eps 1e-12, two
    (ell, sigma^2) settings each (ell log-uniform in [0.05, 2], sigma^2 in [1e-4, 1]), one
    presized lane per problem on 16 lane streams, every result against the exact Kalman
    log-likelihood."""
    import torch
    ninst, per = 64, 2
    un = I.uniform01(3003, ninst)
    sizes = np.round(np.exp(np.log(4096.0) + un * (np.log(262144.0) - np.log(4096.0)))).astype(int)
    assert sizes.max() > 200000 and sizes.min() < 5000
    origin = torch.cuda.Stream()
    pool = [torch.cuda.Stream() for _ in range(16)]
    lanes, keep = [], []
    for i, ni in enumerate(sizes):
        x, y = I.workload_1d(int(ni), 3100 + i)
        ell, s2 = settings(per, 3300 + i)
        h = H.Hodlr(x, "matern52", [ell[0], 1.0], s2[0], 128, 1e-12, precision=precision,
                    stream=pool[i % len(pool)].cuda_stream)
        h.presize(np.full(h.tree()[0], 4, dtype=np.int32))
        theta = torch.from_numpy(np.stack([ell, np.ones(per)], 1).copy()).cuda()
        sig = torch.from_numpy(s2.copy()).cuda()
        yd = torch.from_numpy(y).cuda()
        out = torch.zeros(per, dtype=torch.float64, device="cuda")
        st = torch.full((per,), -1, dtype=torch.int32, device="cuda")
        lanes.append(H.hodlr_batch_lane(h._ctx, theta.data_ptr(), sig.data_ptr(), yd.data_ptr(),
                                        out.data_ptr(), st.data_ptr(), 0, 1, per))
        keep.append((h, x, y, ell, s2, theta, sig, yd, out, st))
    torch.cuda.synchronize()
    assert H.hodlr_loglik_batched(lanes, origin.cuda_stream) == H.HODLR_OK
    torch.cuda.synchronize()
    worst = 0.0
    for h, x, y, ell, s2, theta, sig, yd, out, st in keep:
        assert (st.cpu().numpy() == 0).all()
        got = out.cpu().numpy()
        for b in range(per):
            k = kalman_loglik(x, y, 5, ell[b], s2[b])
            e = abs(got[b] - k) / abs(k)
            worst = max(worst, e)
            assert e <= 1e-9, (len(y), ell[b], s2[b], got[b], k)
        h.close()
    print(f"uneven Matern-5/2 instances, precision {precision}: worst rel. error {worst:.2e}")


def test_batched_lanes_sharing_streams(H):
    """Ten problems on three lane streams (lanes on one stream run one after another)."""
    import torch
    origin = torch.cuda.Stream()
    pool = [torch.cuda.Stream() for _ in range(3)]
    nset = 2
    lanes, keep = [], []
    for i in range(10):
        n = 3000 + 1700 * i
        x, y = I.workload_1d(n, 1200 + i)
        ell, s2 = settings(nset, 400 + i)
        h = H.Hodlr(x, "exp", [ell[0], 1.0], s2[0], 128, 1e-12,
                    stream=pool[i % 3].cuda_stream)
        h.presize(np.full(h.tree()[0], 2, dtype=np.int32))
        theta = torch.from_numpy(np.stack([ell, np.ones(nset)], 1).copy()).cuda()
        sig = torch.from_numpy(s2.copy()).cuda()
        yd = torch.from_numpy(y).cuda()
        out = torch.zeros(nset, dtype=torch.float64, device="cuda")
        st = torch.full((nset,), -1, dtype=torch.int32, device="cuda")
        lanes.append(H.hodlr_batch_lane(h._ctx, theta.data_ptr(), sig.data_ptr(), yd.data_ptr(),
                                        out.data_ptr(), st.data_ptr(), 0, 1, nset))
        keep.append((h, x, y, ell, s2, theta, sig, yd, out, st))
    torch.cuda.synchronize()
    assert H.hodlr_loglik_batched(lanes, origin.cuda_stream) == H.HODLR_OK
    torch.cuda.synchronize()
    for h, x, y, ell, s2, theta, sig, yd, out, st in keep:
        assert (st.cpu().numpy() == 0).all()
        got = out.cpu().numpy()
        for b in range(nset):
            r = H.Hodlr(x, "exp", [ell[b], 1.0], s2[b], 128, 1e-12).loglik(y)
            assert abs(got[b] - r) <= 1e-12 * abs(r)


def test_batched_rejects_bad_lanes(H):
    import torch
    x, y = I.workload_1d(4096, 1020)
    s = torch.cuda.Stream()
    h = H.Hodlr(x, "exp", [0.2, 1.0], 0.01, 64, 1e-12, stream=s.cuda_stream)  # not presized
    theta = torch.ones((2, 2), dtype=torch.float64, device="cuda")
    sig = torch.ones(2, dtype=torch.float64, device="cuda")
    yd = torch.from_numpy(y).cuda()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    lane = H.hodlr_batch_lane(h._ctx, theta.data_ptr(), sig.data_ptr(), yd.data_ptr(),
                              out.data_ptr(), None, 0, 1, 2)
    origin = torch.cuda.Stream()
    assert H.hodlr_loglik_batched([lane], origin.cuda_stream) == H.HODLR_EINVAL
    h.presize(np.full(h.tree()[0], 2, dtype=np.int32))
    assert H.hodlr_loglik_batched([lane], s.cuda_stream) == H.HODLR_EINVAL  # origin = lane stream
    assert "differ from the caller" in H.hodlr_last_error(h._ctx)
    assert H.hodlr_loglik_batched([lane, lane], origin.cuda_stream) == H.HODLR_EINVAL
    assert "two lanes" in H.hodlr_last_error(h._ctx)


def test_batched_lanes_of_both_forms_in_one_call(H):
    """One batched call whose lanes mix the FP64 and the mixed form (two persistent leaf
    launches per round, one per form) and uneven sizes, including a problem that is a
    single leaf: every result equals the adaptive evaluation of its own form."""
    import torch
    origin = torch.cuda.Stream()
    specs = [(120, 0), (5000, 1), (20000, 0), (33000, 1), (9000, 1), (70000, 0)]
    nset = 3
    lanes, keep = [], []
    for i, (n, prec) in enumerate(specs):
        x, y = I.workload_1d(n, 1300 + i)
        ell, s2 = settings(nset, 500 + i)
        h = H.Hodlr(x, "matern32", [ell[0], 1.0], s2[0], 128, 1e-12, precision=prec,
                    stream=torch.cuda.Stream().cuda_stream)
        h.presize(np.full(max(h.tree()[0], 1), 3, dtype=np.int32)[:h.tree()[0]])
        theta = torch.from_numpy(np.stack([ell, np.ones(nset)], 1).copy()).cuda()
        sig = torch.from_numpy(s2.copy()).cuda()
        yd = torch.from_numpy(y).cuda()
        out = torch.zeros(nset, dtype=torch.float64, device="cuda")
        st = torch.full((nset,), -1, dtype=torch.int32, device="cuda")
        lanes.append(H.hodlr_batch_lane(h._ctx, theta.data_ptr(), sig.data_ptr(), yd.data_ptr(),
                                        out.data_ptr(), st.data_ptr(), 0, 1, nset))
        keep.append((h, x, y, ell, s2, prec, theta, sig, yd, out, st))
    torch.cuda.synchronize()
    assert H.hodlr_loglik_batched(lanes, origin.cuda_stream) == H.HODLR_OK
    torch.cuda.synchronize()
    for h, x, y, ell, s2, prec, theta, sig, yd, out, st in keep:
        assert (st.cpu().numpy() == 0).all()
        got = out.cpu().numpy()
        for b in range(nset):
            r = H.Hodlr(x, "matern32", [ell[b], 1.0], s2[b], 128, 1e-12, precision=prec).loglik(y)
            assert abs(got[b] - r) <= 1e-12 * abs(r), (len(y), prec, b, got[b], r)
            k = kalman_loglik(x, y, 3, ell[b], s2[b])
            assert abs(got[b] - k) <= 1e-9 * abs(k), (len(y), prec, b, got[b], k)
