"""Parity of the CUDA path (through the C ABI) with the CPU oracle on the same seeded inputs.

Tolerances: the FP64 path is held to relative 1e-10 on log det and log-likelihood and to
1e-10 relative residual where the configuration allows it (the small squared-exponential
case reaches 1.0e-10 at eps = 1e-12 in the oracle itself, so it is bounded at 2e-10).
Integer results (the point permutation, exact ranks) are compared bit for bit.
"""
import numpy as np
import pytest

import oracle as O
from paper_1403_6015_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch  # noqa: F401
    from paper_1403_6015_gb300 import build_lib, hodlr
    build_lib.build()
    hodlr.load()
    return hodlr


def rel(a, b):
    return abs(a - b) / abs(b)


def dense_C(x, kern, th, s2):
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
    r = np.sqrt(((x[:, None, :] - x[None, :, :]) ** 2).sum(-1))
    return O.kernel_values(kern, r.ravel(), th[0], th[1]).reshape(r.shape) + s2 * np.eye(len(x))


# ------------------------------------------------------------------ ordering -------------

# 2^17 points fill exactly one tile of the radix sort's digit-count scan (256 counts per
# 4096 keys, 8192 counts per tile); 405 561 and 2^20 span 3.1 and 8 tiles.
@pytest.mark.parametrize("n,leaf", [(1, 8), (100, 8), (4097, 64), (1 << 17, 128), (405561, 128),
                                    (1 << 20, 128)])
def test_sort_1d_bit_exact(H, n, leaf):
    x, _ = I.workload_1d(n, 7 + n)
    if n > 10:
        x[5] = x[3]  # a tie, broken by the caller's index
    h = H.Hodlr(x, "exp", [0.2, 1.0], 0.01, leaf, 1e-12)
    kappa, perm = h.tree()
    assert kappa == O.kappa(n, leaf)
    np.testing.assert_array_equal(perm, O.tree_order(x, leaf))


@pytest.mark.parametrize("n,leaf", [(50, 8), (3001, 20), (1 << 15, 64), (300007, 128)])
def test_sort_2d_kd_bit_exact(H, n, leaf):
    x, _ = I.workload_2d(n, 11 + n)
    h = H.Hodlr(x, "se", [0.3, 1.0], 0.01, leaf, 1e-8, allow_rank_cap=True)
    _, perm = h.tree()
    np.testing.assert_array_equal(perm, O.tree_order(x, leaf))


# ------------------------------------------------------------------ compression ----------

@pytest.mark.parametrize("kern,rank", [("exp", 1), ("matern32", 2), ("matern52", 3)])
def test_exact_ranks_match(H, kern, rank):
    """1-D exponential / Matern-3/2 / Matern-5/2 blocks have exact ranks 1 / 2 / 3. At
    eps = 1e-10 the next ACA term (rounding noise) is far below the tolerance, so GPU and
    oracle ranks must agree exactly; at eps = 1e-12 that noise term (about 1e-12 of the
    block for Matern-5/2) may or may not be kept, depending on the last bit of exp(), so
    either rank is correct there."""
    x, _ = I.workload_1d(20000, 51)
    h = H.Hodlr(x, kern, [0.1, 1.0], 0.01, 64, 1e-10)
    r = h.ranks()
    ref = O.Hodlr(x, kern, [0.1, 1.0], 0.01, 64, 1e-10).ranks()
    np.testing.assert_array_equal(r, ref)
    assert set(r.tolist()) == {rank}
    r12 = H.Hodlr(x, kern, [0.1, 1.0], 0.01, 64, 1e-12).ranks()
    assert set(r12.tolist()) <= {rank, rank + 1}
    assert (r12 == rank).mean() > 0.95


def test_se_ranks_close_to_oracle(H):
    x, _ = I.workload_small_se()
    r = H.Hodlr(x, "se", [0.5, 1.0], 0.1, 64, 1e-12).ranks()
    ref = O.Hodlr(x, "se", [0.5, 1.0], 0.1, 64, 1e-12).ranks()
    assert np.abs(r.astype(int) - ref.astype(int)).max() <= 1


# ------------------------------------------------------------------ whole method ---------

def test_small_se_workload(H):
    """n=4096, SE ell=0.5, sigma^2=0.1, leaf 64, eps=1e-12 against O1 dense and O2."""
    x, y = I.workload_small_se()
    th, s2 = [0.5, 1.0], 0.1
    sol_d, ld_d = O.dense_solve(x, "se", th, s2, y)
    h = H.Hodlr(x, "se", th, s2, 64, 1e-12)
    sol = h.factor_solve(y)
    ld = h.logdet()
    assert rel(ld, ld_d) <= 1e-10
    C = dense_C(x, "se", th, s2)
    assert np.linalg.norm(C @ sol - y) / np.linalg.norm(y) <= 2e-10
    ref = O.Hodlr(x, "se", th, s2, 64, 1e-12)
    sol_o = ref.factor_solve(y)
    assert rel(ld, ref.logdet()) <= 1e-10
    assert np.linalg.norm(sol - sol_o) / np.linalg.norm(sol_o) <= 1e-9


CASES = [(1, 8), (7, 8), (8, 8), (9, 8), (100, 7), (257, 16), (1000, 64), (3000, 128),
         (4099, 32), (10000, 100)]


@pytest.mark.parametrize("n,leaf", CASES)
@pytest.mark.parametrize("kern", ["exp", "se", "matern32", "matern52"])
def test_ragged_sizes_vs_dense(H, n, leaf, kern):
    x, y = I.workload_1d(n, 300 + n, nrhs=2)
    th, s2 = [0.3, 1.2], 0.05
    h = H.Hodlr(x, kern, th, s2, leaf, 1e-13)
    sol = h.factor_solve(y)
    if n <= 4500:
        sol_d, ld_d = O.dense_solve(x, kern, th, s2, y)
        assert abs(h.logdet() - ld_d) <= 1e-10 * max(1.0, abs(ld_d))
        np.testing.assert_allclose(sol, sol_d, rtol=0, atol=1e-8 * np.abs(sol_d).max())
    ref = O.Hodlr(x, kern, th, s2, leaf, 1e-13)
    sol_o = ref.factor_solve(y)
    assert abs(h.logdet() - ref.logdet()) <= 1e-10 * max(1.0, abs(ref.logdet()))
    np.testing.assert_allclose(sol, sol_o, rtol=0, atol=1e-9 * np.abs(sol_o).max())


def test_2d_vs_dense(H):
    """2-D points (kd ordering), SE ell=0.5: block ranks up to 57 at eps=1e-12, under the
    GPU's per-block cap of 64."""
    n = 3000
    x, y = I.workload_2d(n, 91)
    th, s2 = [0.5, 1.0], 0.01
    h = H.Hodlr(x, "se", th, s2, 32, 1e-12)
    sol = h.factor_solve(y)
    sol_d, ld_d = O.dense_solve(x, "se", th, s2, y)
    assert rel(h.logdet(), ld_d) <= 1e-10
    C = dense_C(x, "se", th, s2)
    # cond(C) ~ 2e5 here, so the residual of the method at eps=1e-12 is ~2e-9 (the oracle
    # reaches 2.3e-9 itself): bound the GPU by the oracle's residual
    ref = O.Hodlr(x, "se", th, s2, 32, 1e-12)
    res_o = np.linalg.norm(C @ ref.factor_solve(y) - y) / np.linalg.norm(y)
    res = np.linalg.norm(C @ sol - y) / np.linalg.norm(y)
    assert res <= 2.0 * res_o + 1e-12


@pytest.mark.parametrize("nrhs", [1, 3, 16, 21])
def test_standalone_solve_matches_fused(H, nrhs):
    x, y = I.workload_1d(5000, 41, nrhs=nrhs)
    th, s2 = [0.2, 1.0], 0.01
    Y = y.reshape(5000, -1)
    h = H.Hodlr(x, "matern52", th, s2, 64, 1e-12)
    h.factor()
    sol = h.solve(Y)
    ref = O.Hodlr(x, "matern52", th, s2, 64, 1e-12)
    ref.factor()
    sol_o = ref.solve(Y)
    np.testing.assert_allclose(sol, sol_o, rtol=0, atol=1e-9 * np.abs(sol_o).max())
    h2 = H.Hodlr(x, "matern52", th, s2, 64, 1e-12)
    if nrhs <= 16:
        np.testing.assert_allclose(h2.factor_solve(Y), sol, rtol=0, atol=1e-11 * np.abs(sol).max())


def test_loglik_and_device_pointers(H):
    import torch
    n = 20000
    x, y = I.workload_1d(n, 61)
    th, s2 = [0.1, 1.0], 1e-2
    ref = O.Hodlr(x, "matern32", th, s2, 128, 1e-12)
    ll_o = ref.loglik(y)
    h = H.Hodlr(torch.from_numpy(x).cuda(), "matern32", th, s2, 128, 1e-12)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    h.loglik(torch.from_numpy(y).cuda(), out=out)
    assert rel(float(out.item()), ll_o) <= 1e-10
    # second call reuses the factors (standalone solve path)
    out2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    h.loglik(torch.from_numpy(y).cuda(), out=out2)
    assert rel(float(out2.item()), ll_o) <= 1e-10
    xs = h.solve(torch.from_numpy(y).cuda()).cpu().numpy()
    np.testing.assert_allclose(xs, ref.solve(y), rtol=0, atol=1e-9 * np.abs(xs).max())


def test_matvec_matches_oracle(H):
    n = 6000
    x, y = I.workload_1d(n, 71)
    th, s2 = [0.3, 1.0], 0.01
    h = H.Hodlr(x, "se", th, s2, 64, 1e-12)
    ref = O.Hodlr(x, "se", th, s2, 64, 1e-12)
    mv = h.matvec(y)
    mo = ref.matvec(y)
    np.testing.assert_allclose(mv, mo, rtol=0, atol=1e-10 * np.abs(mo).max())


def test_rebuild_matches_fresh_build(H):
    x, y = I.workload_1d(8000, 81)
    h = H.Hodlr(x, "matern32", [0.2, 1.0], 0.01, 64, 1e-12)
    h.factor()
    h.rebuild([0.05, 2.0], 0.3)
    sol = h.factor_solve(y)
    ref = O.Hodlr(x, "matern32", [0.05, 2.0], 0.3, 64, 1e-12)
    sol_o = ref.factor_solve(y)
    assert rel(h.logdet(), ref.logdet()) <= 1e-10
    np.testing.assert_allclose(sol, sol_o, rtol=0, atol=1e-9 * np.abs(sol_o).max())


def test_deterministic(H):
    x, y = I.workload_1d(30000, 82)
    vals = []
    for _ in range(2):
        h = H.Hodlr(x, "se", [0.05, 1.0], 0.01, 128, 1e-10)
        vals.append(h.loglik(y))
    assert vals[0] == vals[1]


# ------------------------------------------------------------------ errors ---------------

def test_error_codes(H):
    x, y = I.workload_1d(500, 83)
    with pytest.raises(H.HodlrError) as e:
        H.Hodlr(x, "exp", [0.2, 1.0], -1.0, 32, 1e-12)
    assert e.value.status == H.HODLR_EINVAL
    with pytest.raises(H.HodlrError):
        H.Hodlr(x, "exp", [0.2, 1.0], 0.1, 200, 1e-12)
    bad = x.copy()
    bad[10] = np.nan
    with pytest.raises(H.HodlrError):
        H.Hodlr(bad, "exp", [0.2, 1.0], 0.1, 32, 1e-12)
    h = H.Hodlr(x, "exp", [0.2, 1.0], 0.1, 32, 1e-12)
    with pytest.raises(H.HodlrError) as e:
        h.solve(y)
    assert e.value.status == H.HODLR_ESTATE
    with pytest.raises(H.HodlrError) as e:
        h.logdet()
    assert e.value.status == H.HODLR_ESTATE
    h.factor()
    with pytest.raises(H.HodlrError) as e:
        h.factor()
    assert e.value.status == H.HODLR_ESTATE


def test_not_spd_reported(H):
    # two identical points and no noise: the leaf Cholesky meets an exactly zero pivot
    x = np.linspace(-1, 1, 64)
    x[1] = x[0]
    h = H.Hodlr(x, "se", [0.3, 1.0], 0.0, 64, 1e-12)
    with pytest.raises(H.HodlrError) as e:
        h.factor()
    assert e.value.status == H.HODLR_ENOTSPD


def test_rank_cap_reported(H):
    x, _ = I.workload_1d(2000, 84)
    with pytest.raises(H.HodlrError) as e:
        H.Hodlr(x, "se", [0.5, 1.0], 0.1, 16, 1e-14, max_rank=2)
    assert e.value.status == H.HODLR_ERANK
    h = H.Hodlr(x, "se", [0.5, 1.0], 0.1, 16, 1e-14, max_rank=2, allow_rank_cap=True)
    assert h.ranks().max() == 2


# ------------------------------------------------------------------ scale ----------------

@pytest.mark.parametrize("n", [1 << 16, 1 << 20])
def test_exponential_vs_ou_closed_form(H, n):
    """The exponential kernel (ell=0.2, sigma^2=1e-2, leaf 128, eps=1e-12) at up to 2^20
    points against the Ornstein-Uhlenbeck closed form: log det and the full solution."""
    x, y = I.workload_1d(n, 1001)
    th, s2 = [0.2, 1.0], 1e-2
    h = H.Hodlr(x, "exp", th, s2, 128, 1e-12)
    sol = h.factor_solve(y)
    _, perm = h.tree()
    sol_c, ld_c = O.ou_closed_form(x[perm, 0], th[0], th[1], s2, y[perm])
    assert rel(h.logdet(), ld_c) <= 1e-10
    err = np.linalg.norm(sol[perm] - sol_c) / np.linalg.norm(sol_c)
    assert err <= 1e-9


@pytest.mark.parametrize("n", [1 << 16, 1 << 20])
def test_matern32_vs_kalman_full_size(H, n):
    """Matern-3/2 (ell=0.1, sigma^2=1e-2, leaf 128, eps=1e-12): log det and y^T C^-1 y from
    the Kalman filter, and exact residual rows C x - y at sampled rows (O(n) each)."""
    x, y = I.workload_1d(n, 1001)
    th, s2 = [0.1, 1.0], 1e-2
    h = H.Hodlr(x, "matern32", th, s2, 128, 1e-12)
    sol = h.factor_solve(y)
    _, perm = h.tree()
    ldk, q = O.matern_kalman(x[perm, 0], 3, th[0], th[1], s2, y[perm])
    assert rel(h.logdet(), ldk) <= 1e-10
    assert rel(float(y @ sol), q) <= 1e-10
    rows = np.unique(np.linspace(0, n - 1, 64).astype(np.int64))
    Cx = O.dense_matvec_rows(x, "matern32", th, s2, sol, rows)
    res = np.abs(Cx - y[rows]).max() / np.abs(y).max()
    assert res <= 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_nrhs16_full_size_every_column(H, precision):
    """The fused factor-solve with 16 right-hand sides at n = 2^20 (the exponential kernel,
    ell=0.2, sigma^2=1e-2, leaf 128, eps=1e-12), in both forms: every column of C^-1 Y
    against the Ornstein-Uhlenbeck closed form, and the log det."""
    n, nrhs = 1 << 20, 16
    x, Y = I.workload_1d(n, 1001, nrhs)
    th, s2 = [0.2, 1.0], 1e-2
    h = H.Hodlr(x, "exp", th, s2, 128, 1e-12, max_nrhs=nrhs, precision=precision)
    sol = h.factor_solve(Y)
    assert sol.shape == (n, nrhs)
    _, perm = h.tree()
    sol_c, ld_c = O.ou_closed_form(x[perm, 0], th[0], th[1], s2, Y[perm])
    assert rel(h.logdet(), ld_c) <= 1e-10
    for c in range(nrhs):
        err = np.linalg.norm(sol[perm, c] - sol_c[:, c]) / np.linalg.norm(sol_c[:, c])
        assert err <= 1e-9, (c, err)


@pytest.mark.parametrize("kern,ell", [("exp", 0.002), ("se", 0.003), ("matern32", 0.02), ("matern52", 0.02)])
def test_fp64_covariance_entries_to_the_last_bits(H, kern, ell):
    """The FP64 covariances evaluate exp by a table-driven method of their own (Tang's, one
    unit in the last place). On a single-leaf problem C v is the dense product of those
    entries with v, so it must match the oracle's dense rows (libm exp, compensated sums) to
    a few units of roundoff in sum |C_ij v_j|. The short length scales take the arguments
    of exp from 0 down past -745, through the subnormal range into underflow."""
    n = 128
    x = np.sort(I.uniform_points(n, 1, -1.0, 1.0, 2200 + len(kern)).reshape(-1))
    v = I.normal(n, 2201)
    s2 = 1e-2
    h = H.Hodlr(x, kern, [ell, 1.0], s2, 128, 1e-12)
    assert h.tree()[0] == 0  # one leaf: every entry is evaluated, nothing compressed
    got = h.matvec(v)
    ref = O.dense_matvec_rows(x, kern, [ell, 1.0], s2, v, np.arange(n))
    C = O.kernel_values(kern, np.abs(x[:, None] - x[None, :]), ell, 1.0)
    scale = np.abs(C) @ np.abs(v) + s2 * np.abs(v)
    assert np.all(np.abs(got - ref) <= 8 * 2.0 ** -52 * scale), np.max(np.abs(got - ref) / scale)
