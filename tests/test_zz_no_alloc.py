"""The allocation-free entry point (hodlr_loglik_small_noalloc) against the regular one.

Callers that cannot allocate device memory while they evaluate (a fixed memory budget, a
graph without allocation nodes) use hodlr_loglik_small_noalloc for problems of one leaf
block. Its result must equal the regular hodlr_build + hodlr_loglik path and the oracle's
dense Cholesky on the same input, call after call, since every call reuses the same fixed
scratch array, and repeated calls must leave the device's memory untouched. This file
is collected last so that a stopping run has already run every other test.
"""
import ctypes

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


@pytest.mark.parametrize("n,d,kern", [(100, 1, "matern32"), (128, 2, "se"), (1, 1, "exp"),
                                      (57, 1, "matern52"), (128, 3, "matern52")])
def test_noalloc_matches_regular_entry_twice(H, n, d, kern):
    import torch
    x = I.uniform_points(n, d, -1.0, 1.0, 500 + n) if d != 2 else I.workload_2d(n, 500 + n)[0]
    y = I.normal(n, 600 + n)
    th, s2 = [0.3, 1.1], 0.05
    ref = H.Hodlr(x, kern, th, s2, 128, 1e-12).loglik(y)  # regular path (one leaf)
    # the plain definition: dense Cholesky in the oracle
    sol, ld = O.dense_solve(x, kern, th, s2, y)
    dense = -0.5 * float(y @ sol) - 0.5 * ld - 0.5 * n * np.log(2.0 * np.pi)
    assert abs(ref - dense) <= 1e-10 * abs(dense), (ref, dense)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.from_numpy(y).cuda()
    for _ in range(2):
        out = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
        st = H.hodlr_loglik_small_noalloc(xd.data_ptr(), n, d, H.KERNELS[kern], th, s2,
                                          yd.data_ptr(), out.data_ptr(), None)
        assert st == H.HODLR_OK
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= 1e-10 * abs(ref), (got, ref)
        assert abs(got - dense) <= 1e-10 * abs(dense), (got, dense)


def test_noalloc_allocates_nothing(H):
    """After one warm-up call (which may load the kernels' code), further calls change
    neither the device's free memory nor torch's allocator."""
    import torch
    n, kern, th, s2 = 120, "matern52", [0.4, 1.0], 0.02
    x = I.uniform_points(n, 1, -1.0, 1.0, 777)
    y = I.normal(n, 778)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.from_numpy(y).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    args = (xd.data_ptr(), n, 1, H.KERNELS[kern], th, s2, yd.data_ptr(), out.data_ptr(), None)
    assert H.hodlr_loglik_small_noalloc(*args) == H.HODLR_OK
    torch.cuda.synchronize()
    first = float(out.item())
    free0, _ = torch.cuda.mem_get_info()
    torch0 = torch.cuda.memory_allocated()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(5):
        assert H.hodlr_loglik_small_noalloc(*args) == H.HODLR_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == torch0
    assert torch.cuda.memory_reserved() == reserved0
    assert float(out.item()) == first


def test_noalloc_rejects_oversize_and_host_pointers(H):
    import torch
    n = 129
    xd = torch.zeros(n, dtype=torch.float64, device="cuda")
    yd = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = H.hodlr_loglik_small_noalloc(xd.data_ptr(), n, 1, 0, [0.3, 1.0], 0.1, yd.data_ptr(),
                                      out.data_ptr(), None)
    assert st == H.HODLR_EINVAL
    xh = np.linspace(0, 1, 10)
    yh = np.ones(10)
    oh = np.zeros(1)
    st = H.hodlr_loglik_small_noalloc(xh.ctypes.data, 10, 1, 0, [0.3, 1.0], 0.1, yh.ctypes.data,
                                      oh.ctypes.data, None)
    assert st == H.HODLR_EINVAL
    # the radial covariances are not served by this entry
    st = H.hodlr_loglik_small_noalloc(xd.data_ptr(), 10, 1, H.KERNELS["imq"], [0.3, 1.0], 0.1,
                                      yd.data_ptr(), out.data_ptr(), None)
    assert st == H.HODLR_EINVAL


def test_noalloc_not_spd_gives_nan(H):
    import torch
    x = np.linspace(-1, 1, 64)
    x[1] = x[0]
    xd = torch.from_numpy(x).cuda()
    yd = torch.ones(64, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = H.hodlr_loglik_small_noalloc(xd.data_ptr(), 64, 1, 1, [0.3, 1.0], 0.0, yd.data_ptr(),
                                      out.data_ptr(), None)
    assert st == H.HODLR_OK
    torch.cuda.synchronize()
    assert np.isnan(float(out.item()))
