"""Presized (synchronisation-free) compression and the graph-replayed hyperparameter sweep.

The sweep evaluates many (ell, sigma^2) settings on one set of points, as in
hyperparameter adaptation (Sec. 2.5); each setting's log-likelihood must equal the one the
adaptive path computes for that setting alone, and the Kalman filter's exact value.
"""
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


def settings(nset, seed):
    """ell log-uniform in [0.05, 2], sigma^2 log-uniform in [1e-4, 1]."""
    u = I.uniform01(seed, 2 * nset)
    ell = np.exp(np.log(0.05) + u[:nset] * (np.log(2.0) - np.log(0.05)))
    s2 = np.exp(np.log(1e-4) + u[nset:] * (np.log(1.0) - np.log(1e-4)))
    return ell, s2


def rel(a, b):
    return abs(a - b) / abs(b)


@pytest.mark.parametrize("precision", [0, 1])
def test_presized_matches_adaptive(H, precision):
    import torch
    n = 1 << 14
    x, y = I.workload_1d(n, 1004)
    ell, s2 = settings(6, 77)
    stream = torch.cuda.Stream()
    ref = [H.Hodlr(x, "matern52", [e, 1.0], s, 128, 1e-12, precision=precision).loglik(y)
           for e, s in zip(ell, s2)]
    h = H.Hodlr(x, "matern52", [ell[0], 1.0], s2[0], 128, 1e-12, precision=precision,
                stream=stream.cuda_stream)
    h.presize(np.full(h.tree()[0], 4, dtype=np.int32))
    for e, s, r in zip(ell, s2, ref):
        h.rebuild([e, 1.0], s)
        got = h.loglik(y)
        assert rel(got, r) <= 1e-12, (got, r)
    assert h.status_flags() == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_sweep_graph(H, precision):
    import torch
    n, nset = 1 << 16, 24
    x, y = I.workload_1d(n, 1004)
    ell, s2 = settings(nset, 78)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        xd = torch.from_numpy(x).cuda()
        yd = torch.from_numpy(y).cuda()
        theta = torch.from_numpy(np.stack([ell, np.ones(nset)], 1).copy()).cuda()
        sig = torch.from_numpy(s2.copy()).cuda()
        status = torch.full((nset,), -1, dtype=torch.int32, device="cuda")
    stream.synchronize()
    h = H.Hodlr(xd, "matern52", [ell[0], 1.0], s2[0], 128, 1e-12, precision=precision,
                stream=stream.cuda_stream)
    h.presize(np.full(h.tree()[0], 4, dtype=np.int32))
    out = h.loglik_sweep(theta, sig, yd, status=status)
    stream.synchronize()
    got = out.cpu().numpy()
    assert (status.cpu().numpy() == 0).all()
    # every setting against an adaptive evaluation on its own
    for b in [0, 1, 7, nset - 1]:
        r = H.Hodlr(x, "matern52", [ell[b], 1.0], s2[b], 128, 1e-12, precision=precision).loglik(y)
        assert rel(got[b], r) <= 1e-12
    # against the exact Kalman log-likelihood (loosest where cond(C) is largest)
    _, perm = h.tree()
    for b in range(nset):
        ld, q = O.matern_kalman(x[perm, 0], 5, ell[b], 1.0, s2[b], y[perm])
        ll = -0.5 * q - 0.5 * ld - 0.5 * n * np.log(2 * np.pi)
        assert rel(got[b], ll) <= 1e-9, (b, ell[b], s2[b], got[b], ll)
    # a second sweep replays the captured graph: identical results
    out2 = h.loglik_sweep(theta, sig, yd, status=status)
    stream.synchronize()
    np.testing.assert_array_equal(out2.cpu().numpy(), got)


def test_sweep_flags_undersized_presize(H):
    import torch
    n, nset = 1 << 14, 4
    x, y = I.workload_1d(n, 1005)
    ell, s2 = settings(nset, 79)
    stream = torch.cuda.Stream()
    h = H.Hodlr(x, "matern52", [ell[0], 1.0], s2[0], 128, 1e-12, stream=stream.cuda_stream)
    h.presize(np.full(h.tree()[0], 1, dtype=np.int32))  # Matern-5/2 blocks need rank 3
    theta = torch.from_numpy(np.stack([ell, np.ones(nset)], 1).copy()).cuda()
    sig = torch.from_numpy(s2.copy()).cuda()
    yd = torch.from_numpy(y).cuda()
    status = torch.zeros(nset, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    h.loglik_sweep(theta, sig, yd, status=status)
    stream.synchronize()
    assert ((status.cpu().numpy() & 2) != 0).all()


def test_presize_rejects_bad_input(H):
    x, _ = I.workload_1d(4096, 1006)
    h = H.Hodlr(x, "exp", [0.2, 1.0], 0.01, 64, 1e-12)
    with pytest.raises(H.HodlrError):
        h.presize(np.ones(3, dtype=np.int32))  # kappa is 6
    with pytest.raises(H.HodlrError):
        h.presize(np.full(6, 64, dtype=np.int32))  # rank + 1 must fit max_rank
    h.presize(None)


@pytest.mark.parametrize("precision", [0, 1])
def test_sweep_graph_general_case(H, precision):
    """The captured sweep on a problem the specialised compression kernels do not cover
    (3-D points, inverse multiquadric): the general instantiation is chosen at launch and
    captured with the rest; every setting equals its adaptive evaluation."""
    import torch
    n, nset = 1 << 13, 6
    x, y = I.workload_3d(n, 1007)
    y = np.ascontiguousarray(y).reshape(-1)
    ell = np.array([2.0, 2.2, 2.4, 2.6, 2.8, 3.0])
    s2 = np.array([0.5, 0.3, 0.2, 0.2, 0.1, 0.1])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        xd = torch.from_numpy(x).cuda()
        yd = torch.from_numpy(y).cuda()
        theta = torch.from_numpy(np.stack([ell, np.ones(nset)], 1).copy()).cuda()
        sig = torch.from_numpy(s2.copy()).cuda()
        status = torch.full((nset,), -1, dtype=torch.int32, device="cuda")
    stream.synchronize()
    h = H.Hodlr(xd, "imq", [ell[0], 1.0], s2[0], 64, 1e-8, max_rank=256, precision=precision,
                stream=stream.cuda_stream)
    kappa, _ = h.tree()
    r = h.ranks()
    prof = np.array([r[(1 << j) - 1:(1 << (j + 1)) - 1].max() for j in range(kappa)]) + 4
    h.presize(np.minimum(prof, 255).astype(np.int32))
    out = h.loglik_sweep(theta, sig, yd, status=status)
    stream.synchronize()
    assert (status.cpu().numpy() == 0).all()
    got = out.cpu().numpy()
    for b in range(nset):
        ref = H.Hodlr(x, "imq", [ell[b], 1.0], s2[b], 64, 1e-8, max_rank=256,
                      precision=precision).loglik(y)
        assert rel(got[b], ref) <= 1e-12, (b, got[b], ref)


@pytest.mark.parametrize("precision", [0, 1])
def test_presized_node_step_at_rank_39(H, precision):
    """A node matrix of rank 39 takes 4 x 39^2 x 8 = 48,672 bytes of dynamic shared
    memory: with the kernel's static arrays just over the 48 KB a launch may use without
    opting in. Presized padding to 39 (fused sweep), and to 67 at the top with 39 below
    (unfused sweep), must still give the adaptive log-likelihood."""
    x, y = I.workload_1d(1 << 14, 1008)
    th, s2 = [0.3, 1.0], 1e-2
    ref = H.Hodlr(x, "se", th, s2, 64, 1e-12, max_rank=128, precision=precision).loglik(y)
    h = H.Hodlr(x, "se", th, s2, 64, 1e-12, max_rank=128, precision=precision)
    kappa, _ = h.tree()
    for prof in ([39] * kappa, [67] + [39] * (kappa - 1)):
        h.presize(np.array(prof, dtype=np.int32))
        h.rebuild(th, s2)
        got = h.loglik(y)
        assert h.status_flags() == 0
        assert rel(got, ref) <= 1e-12, (prof[:2], got, ref)
