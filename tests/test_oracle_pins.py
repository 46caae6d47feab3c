"""Pins for the CPU oracle: each check compares it with something other than itself.

Kinds of pin used (no GPU needed):
  - published test vectors (splitmix64, tests/golden/splitmix64.txt);
  - library routines of a different algorithm (LAPACK via numpy/scipy, Bessel K_nu);
  - closed forms (Ornstein-Uhlenbeck tridiagonal inverse) and the Kalman filter, each an
    independent route to C^-1 y and log det C;
  - identities from the paper (Sylvester's determinant theorem, Sec. 4; the
    Sherman-Morrison-Woodbury formula, Sec. 3.2);
  - exact-rank facts (1-D exponential / Matern-3/2 / Matern-5/2 blocks of disjoint sorted
    sets have rank 1 / 2 / 3) and the truncated SVD (optimal low rank, Sec. 3.1);
  - the paper's claims: results independent of the leaf size (Sec. 5.6) and error
    decreasing with the tolerance.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.special as sps
import scipy.stats as sst

import oracle as O
from paper_1403_6015_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_C(x, kern, theta, s2):
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
    r = np.sqrt(((x[:, None, :] - x[None, :, :]) ** 2).sum(-1))
    th = list(theta) + [1.0] * (3 - len(theta))
    K = O.kernel_values(kern, r.ravel(), *th).reshape(r.shape)
    return K + s2 * np.eye(len(x))


# ---------------------------------------------------------------- inputs ----------------

def test_splitmix64_published_vectors():
    for line in open(os.path.join(GOLDEN, "splitmix64.txt")):
        if line.startswith("#") or not line.strip():
            continue
        seed, *outs = line.split()
        got = I.splitmix64(int(seed), len(outs))
        assert [int(o, 16) for o in outs] == [int(g) for g in got]


def test_inputs_shapes_and_ranges():
    x = I.uniform_points(1000, 2, 0.0, 1.0, 7)
    assert x.shape == (1000, 2) and x.min() >= 0 and x.max() < 1
    g = I.normal(200000, 3)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1) < 0.01
    Y = I.normal(100, 3, 4)
    assert Y.shape == (100, 4) and Y.flags.f_contiguous


# ---------------------------------------------------------------- kernels ---------------

@pytest.mark.parametrize("nu2,name", [(1, "exp"), (3, "matern32"), (5, "matern52")])
def test_matern_closed_forms_match_bessel(nu2, name):
    """Half-integer Matern closed forms equal the Bessel form of Table 1 (with ell)."""
    nu = nu2 / 2.0
    ell = 0.37
    r = np.linspace(1e-3, 3.0, 400)
    z = np.sqrt(2 * nu) * r / ell
    bessel = z ** nu * sps.kv(nu, z) / (sps.gamma(nu) * 2 ** (nu - 1))
    got = O.kernel_values(name, r, ell, 1.0)
    np.testing.assert_allclose(got, bessel, rtol=1e-12, atol=1e-300)
    assert O.kernel_values(name, np.zeros(1), ell, 2.5)[0] == 2.5


def test_se_special_values():
    # k(ell) = exp(-1/2), k(0) = a, k(2 ell) = exp(-2)
    v = O.kernel_values("se", np.array([0.0, 0.3, 0.6]), 0.3, 1.7)
    np.testing.assert_allclose(v, 1.7 * np.array([1.0, np.exp(-0.5), np.exp(-2.0)]), rtol=1e-15)


def test_radial_kernels_special_values():
    """Sec. 5's radial functions with the distance in units of ell (a = 1.3, ell = 0.4)."""
    a, ell = 1.3, 0.4
    e = np.e
    # multiquadric sqrt(1 + t^2): 1 at 0, 2 at t = sqrt(3)
    np.testing.assert_allclose(O.kernel_values("mq", np.array([0.0, ell * np.sqrt(3.0)]), ell, a),
                               [a, 2 * a], rtol=1e-15)
    # inverse multiquadric 1/sqrt(1 + t^2): 1/2 at t = sqrt(3)
    np.testing.assert_allclose(O.kernel_values("imq", np.array([0.0, ell * np.sqrt(3.0)]), ell, a),
                               [a, a / 2], rtol=1e-15)
    # biharmonic t^2 log t: 0 at 0 and 1, e^2 at e, -1/e^2 at 1/e, 4 log 2 at 2
    r = ell * np.array([0.0, 1.0, e, 1 / e, 2.0])
    np.testing.assert_allclose(O.kernel_values("biharmonic", r, ell, a),
                               a * np.array([0.0, 0.0, e * e, -1 / e ** 2, 4 * np.log(2.0)]),
                               rtol=1e-14, atol=1e-16)
    # rational quadratic (1 + t^2)^-alpha: 2^-alpha at t = 1, 4^-2.5 = 1/32 at t = sqrt(3)
    np.testing.assert_allclose(O.kernel_values("rq", np.array([0.0, ell, ell * np.sqrt(3.0)]), ell,
                                               a, 2.5),
                               a * np.array([1.0, 2 ** -2.5, 1 / 32]), rtol=1e-15)


def test_radial_kernel_identities():
    r = np.linspace(0.0, 5.0, 301)
    ell, a = 0.7, 1.1
    mq = O.kernel_values("mq", r, ell, a)
    imq = O.kernel_values("imq", r, ell, a)
    np.testing.assert_allclose(mq * imq, a * a, rtol=1e-15)
    # the inverse multiquadric is the rational quadratic with alpha = 1/2
    np.testing.assert_allclose(O.kernel_values("rq", r, ell, a, 0.5), imq, rtol=1e-15)
    # (1 + r^2 / (2 alpha l^2))^-alpha -> exp(-r^2 / (2 l^2)) as alpha grows (relative
    # error about r^4 / (8 alpha l^4), below 2e-7 for r <= 3)
    l0, big = 0.9, 1e8
    r3 = r[r <= 3.0]
    rq = O.kernel_values("rq", r3, l0 * np.sqrt(2 * big), a, big)
    np.testing.assert_allclose(rq, O.kernel_values("se", r3, l0, a), rtol=3e-7)


def test_radial_kernel_matrix_signatures():
    """Eigenvalue structure fixed by the theory of radial functions: a multiquadric matrix
    of distinct points has exactly one positive eigenvalue (Micchelli 1986); the biharmonic
    r^2 log r is conditionally positive definite of order 2, so at most two of its
    eigenvalues are non-positive; the inverse multiquadric matrix is positive definite.
    Smooth kernels have eigenvalues that decay to the rounding level, so signs are counted
    above 1e-10 of the largest magnitude (LAPACK's eigvalsh)."""
    x = np.sort(I.uniform_points(300, 1, -3.0, 3.0, 41)[:, 0])
    r = np.abs(x[:, None] - x[None, :])

    def ev(kern, rr):
        e = np.linalg.eigvalsh(O.kernel_values(kern, rr.ravel(), 1.0, 1.0).reshape(rr.shape))
        return e / np.abs(e).max()

    e_mq = ev("mq", r)
    assert (e_mq > 1e-10).sum() == 1 and e_mq.max() == 1.0
    assert (e_mq < -1e-10).sum() >= 5
    e_bh = ev("biharmonic", r)
    assert (e_bh < -1e-10).sum() <= 2 and (e_bh > 1e-10).sum() >= 5
    assert np.linalg.eigvalsh(O.kernel_values("imq", r.ravel(), 1.0, 1.0).reshape(r.shape)).min() > -1e-12
    x2 = I.uniform_points(200, 2, -3.0, 3.0, 42)
    r2 = np.sqrt(((x2[:, None, :] - x2[None, :, :]) ** 2).sum(-1))
    e2 = ev("mq", r2)
    assert (e2 > 1e-10).sum() == 1 and (e2 < -1e-10).sum() >= 20


# ---------------------------------------------------------------- O1 dense --------------

@pytest.mark.parametrize("kern", ["exp", "se", "matern32", "matern52"])
@pytest.mark.parametrize("d", [1, 2])
def test_dense_matches_lapack(kern, d):
    n = 300
    x = I.uniform_points(n, d, -1, 1, 11)
    y = I.normal(n, 12, 3)
    th, s2 = [0.4, 1.3], 0.05
    C = dense_C(x, kern, th, s2)
    sol, ld = O.dense_solve(x, kern, th, s2, y)
    sign, ref = np.linalg.slogdet(C)
    assert sign > 0
    assert abs(ld - ref) <= 1e-11 * abs(ref)
    np.testing.assert_allclose(sol, sla.solve(C, y, assume_a="pos"), rtol=1e-9, atol=1e-9)


def test_dense_tiny_cofactor():
    """3x3 determinant by cofactor expansion (no factorization at all)."""
    x = np.array([0.1, -0.4, 0.9])
    C = dense_C(x, "matern32", [0.5, 1.0], 0.2)
    det = (C[0, 0] * (C[1, 1] * C[2, 2] - C[1, 2] * C[2, 1])
           - C[0, 1] * (C[1, 0] * C[2, 2] - C[1, 2] * C[2, 0])
           + C[0, 2] * (C[1, 0] * C[2, 1] - C[1, 1] * C[2, 0]))
    _, ld = O.dense_solve(x, "matern32", [0.5, 1.0], 0.2, np.ones(3))
    assert abs(ld - np.log(det)) < 1e-14


def test_dense_rejects_non_spd():
    # sigma^2 < 0 large enough to make C indefinite
    x = np.linspace(-1, 1, 20)
    with pytest.raises(O.OracleError):
        O.dense_solve(x, "se", [0.3, 1.0], -2.0, np.ones(20))


def test_dense_matvec_rows_exact():
    n = 500
    x = I.uniform_points(n, 1, -1, 1, 5)
    v = I.normal(n, 6)
    C = dense_C(x, "matern52", [0.2, 1.0], 0.01)
    rows = np.array([0, 17, 250, 499])
    np.testing.assert_allclose(O.dense_matvec_rows(x, "matern52", [0.2, 1.0], 0.01, v, rows),
                               (C @ v)[rows], rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------- closed forms ----------

def test_ou_closed_form_vs_dense():
    n = 1500
    x, y = I.workload_1d(n, 21, nrhs=2)
    xs = np.sort(x[:, 0])
    p = np.argsort(x[:, 0], kind="stable")
    th, s2 = [0.2, 1.4], 0.01
    sol_d, ld_d = O.dense_solve(x, "exp", th, s2, y)
    sol_c, ld_c = O.ou_closed_form(xs, th[0], th[1], s2, y[p])
    assert abs(ld_c - ld_d) <= 1e-11 * abs(ld_d)
    np.testing.assert_allclose(sol_c, sol_d[p], rtol=1e-8, atol=1e-8 * np.abs(sol_d).max())


@pytest.mark.parametrize("nu2,name", [(1, "exp"), (3, "matern32"), (5, "matern52")])
def test_kalman_vs_dense(nu2, name):
    n = 1200
    x, y = I.workload_1d(n, 31)
    p = np.argsort(x[:, 0], kind="stable")
    th, s2 = [0.15, 0.8], 0.02
    sol, ld = O.dense_solve(x, name, th, s2, y)
    ldk, q = O.matern_kalman(x[p, 0], nu2, th[0], th[1], s2, y[p])
    assert abs(ldk - ld) <= 1e-10 * abs(ld)
    assert abs(q - y @ sol) <= 1e-9 * abs(q)


def test_loglik_formula_vs_scipy():
    n = 200
    x, y = I.workload_1d(n, 41)
    th, s2 = [0.3, 1.0], 0.1
    C = dense_C(x, "se", th, s2)
    H = O.Hodlr(x, "se", th, s2, 16, 1e-14)
    ref = sst.multivariate_normal(mean=np.zeros(n), cov=C).logpdf(y)
    assert abs(H.loglik(y) - ref) <= 1e-9 * abs(ref)


# ---------------------------------------------------------------- identities ------------

def test_sylvester_identity():
    """det(I_m + A B) = det(I_n + B A) (Sec. 4), through the oracle's LU."""
    rng = np.random.default_rng(0)
    A = rng.standard_normal((80, 5)) * 0.3
    B = rng.standard_normal((5, 80)) * 0.3
    big, s1 = O.lu_logdet(np.eye(80) + A @ B)
    small, s2 = O.lu_logdet(np.eye(5) + B @ A)
    assert s1 == s2 and abs(big - small) < 1e-12
    ref = np.linalg.slogdet(np.eye(80) + A @ B)
    assert abs(big - ref[1]) < 1e-12 and s1 == ref[0]


def test_smw_identity():
    """(A + L S R)^-1 b = A^-1 b - A^-1 L (S^-1 + R A^-1 L)^-1 R A^-1 b (Sec. 3.2)."""
    rng = np.random.default_rng(1)
    m, r = 60, 4
    A = np.eye(m) * 3 + rng.standard_normal((m, m)) * 0.1
    L = rng.standard_normal((m, r))
    S = np.eye(r) + rng.standard_normal((r, r)) * 0.1
    R = rng.standard_normal((r, m))
    b = rng.standard_normal(m)
    direct = O.lu_solve(A + L @ S @ R, b)
    Ainv_b = O.lu_solve(A, b)
    AinvL = np.column_stack([O.lu_solve(A, L[:, k]) for k in range(r)])
    inner = np.linalg.inv(S) + R @ AinvL
    smw = Ainv_b - AinvL @ O.lu_solve(inner, R @ Ainv_b)
    np.testing.assert_allclose(smw, direct, rtol=1e-12, atol=1e-12)


def test_lu_negative_determinant_sign():
    A = np.diag([1.0, -2.0, 3.0])
    ld, sg = O.lu_logdet(A)
    assert sg == -1 and abs(ld - np.log(6.0)) < 1e-15


# ---------------------------------------------------------------- ordering --------------

def test_tree_order_1d_is_stable_sort():
    x = I.uniform_points(5000, 1, -1, 1, 3)
    x[100] = x[200]  # a tie: the lower original index comes first
    np.testing.assert_array_equal(O.tree_order(x, 32), np.argsort(x[:, 0], kind="stable"))


@pytest.mark.parametrize("d", [2, 3])
def test_tree_order_kd_invariant(d):
    """Sec. 3: each split halves its node by point count along dimension depth mod d."""
    n, leaf = 3000, 20
    x = I.uniform_points(n, d, 0, 1, 4)
    perm = O.tree_order(x, leaf)
    assert sorted(perm.tolist()) == list(range(n))
    xs = x[perm]
    kap = O.kappa(n, leaf)

    def check(b, m, depth):
        if depth >= kap:
            return
        dim = depth % d
        ml = m // 2
        assert xs[b:b + ml, dim].max() <= xs[b + ml:b + m, dim].min()
        check(b, ml, depth + 1)
        check(b + ml, m - ml, depth + 1)

    check(0, n, 0)


def test_kappa_reading():
    assert O.kappa(1 << 20, 128) == 13
    assert O.kappa(4096, 64) == 6
    assert O.kappa(100, 128) == 0
    assert O.kappa(129, 128) == 1
    assert O.kappa(4097, 64) == 7


# ---------------------------------------------------------------- compression -----------

@pytest.mark.parametrize("name,rank", [("exp", 1), ("matern32", 2), ("matern52", 3)])
def test_aca_exact_ranks(name, rank):
    """Exact ranks 1 / 2 / 3 at eps = 1e-10 (at 1e-12 the rounding-noise term of a
    Matern-5/2 block sits near the tolerance and is sometimes kept)."""
    x, _ = I.workload_1d(4096, 51)
    H = O.Hodlr(x, name, [0.1, 1.0], 0.01, 64, 1e-10)
    assert set(H.ranks().tolist()) == {rank}


def test_aca_se_error_vs_svd():
    """ACA block error is at the tolerance's scale and its rank is near the SVD eps-rank."""
    n, eps = 1024, 1e-10
    x, _ = I.workload_1d(n, 61)
    th = [0.3, 1.0]
    H = O.Hodlr(x, "se", th, 0.1, 64, eps)
    xs = x[H.perm(), 0]
    for node in range(3):
        (bl, ml), (br, mr) = H.node_range(2 * node + 1), H.node_range(2 * node + 2)
        B = dense_C(xs, "se", th, 0.0)[bl:bl + ml, br:br + mr]
        U, V = H.node_factors(node)
        err = np.linalg.norm(B - U @ V.T) / np.linalg.norm(B)
        assert err <= 100 * eps
        s = np.linalg.svd(B, compute_uv=False)
        svd_rank = int(np.sum(s > eps * s[0]))
        assert svd_rank - 2 <= U.shape[1] <= svd_rank + 4


def test_aca_rank_cap_reports():
    x, _ = I.workload_1d(512, 71)
    with pytest.raises(O.OracleError):
        O.Hodlr(x, "se", [0.5, 1.0], 0.1, 16, 1e-14, max_rank=2)
    H = O.Hodlr(x, "se", [0.5, 1.0], 0.1, 16, 1e-14, max_rank=2, allow_rank_cap=True)
    assert H.status == 4 and H.ranks().max() == 2


# ---------------------------------------------------------------- O2 vs O1 --------------

def rel_residual(x, kern, th, s2, sol, y):
    C = dense_C(x, kern, th, s2)
    return np.linalg.norm(C @ sol - y) / np.linalg.norm(y)


def test_hodlr_small_se_vs_dense():
    """The small squared-exponential workload: n=4096, ell=0.5, sigma^2=0.1, leaf 64."""
    x, y = I.workload_small_se()
    th, s2 = [0.5, 1.0], 0.1
    sol_d, ld_d = O.dense_solve(x, "se", th, s2, y)
    H = O.Hodlr(x, "se", th, s2, 64, 1e-12)
    sol = H.factor_solve(y)
    assert abs(H.logdet() - ld_d) <= 1e-10 * abs(ld_d)
    # ACA meets eps per block; the residual scales as eps |K| |C^-1| (about 1.0e-10 here),
    # so the 1e-10 residual bar is checked at eps = 3e-13 and eps = 1e-12 gets 2e-10.
    assert rel_residual(x, "se", th, s2, sol, y) <= 2e-10
    np.testing.assert_allclose(H.solve(y), sol, rtol=0, atol=1e-12 * np.abs(sol).max())
    H2 = O.Hodlr(x, "se", th, s2, 64, 3e-13)
    assert rel_residual(x, "se", th, s2, H2.factor_solve(y), y) <= 1e-10


def test_aca_far_field_underflow():
    """A block whose rows far from the interface are exactly zero in FP64 (squared-
    exponential, ell = 0.01 on [-1, 1]: exp(-r^2/(2 ell^2)) underflows for r > 0.39): the
    cross starts at the row nearest the split, so the top-level block keeps its rank and
    the log-likelihood matches dense Cholesky (a start far from the split gave rank 0 and
    a 8e-4 error here)."""
    x, y = I.workload_1d(8192, 1002)
    th, s2 = [0.01, 1.0], 1e-2
    H = O.Hodlr(x, "se", th, s2, 64, 1e-12, max_rank=500)
    assert H.ranks()[0] >= 10
    sol_d, ld_d = O.dense_solve(x, "se", th, s2, y)
    ll_d = -0.5 * y @ sol_d - 0.5 * ld_d - 0.5 * len(y) * np.log(2 * np.pi)
    assert abs(H.loglik(y) - ll_d) <= 1e-10 * abs(ll_d)


@pytest.mark.parametrize("n,leaf", [(8, 2), (37, 3), (100, 7), (257, 16), (512, 16)])
@pytest.mark.parametrize("kern", ["exp", "se", "matern32", "matern52"])
def test_hodlr_brute_force_small(n, leaf, kern):
    x, y = I.workload_1d(n, 80 + n)
    th, s2 = [0.3, 1.0], 0.05
    sol_d, ld_d = O.dense_solve(x, kern, th, s2, y)
    H = O.Hodlr(x, kern, th, s2, leaf, 1e-14)
    sol = H.factor_solve(y)
    assert abs(H.logdet() - ld_d) <= 1e-11 * max(1.0, abs(ld_d))
    np.testing.assert_allclose(sol, sol_d, rtol=0, atol=1e-10 * np.abs(sol_d).max())


def test_hodlr_2d_vs_dense():
    n = 1500
    x, y = I.workload_2d(n, 91)
    th, s2 = [0.1, 1.0], 0.01
    sol_d, ld_d = O.dense_solve(x, "se", th, s2, y)
    H = O.Hodlr(x, "se", th, s2, 32, 1e-12, max_rank=1000)
    sol = H.factor_solve(y)
    assert abs(H.logdet() - ld_d) <= 1e-10 * abs(ld_d)
    assert rel_residual(x, "se", th, s2, sol, y) <= 1e-9


@pytest.mark.parametrize("kern,ell,eps,tol", [("se", 1.0, 1e-12, 1e-10), ("matern52", 0.5, 1e-10, 1e-9)])
def test_hodlr_3d_vs_dense(kern, ell, eps, tol):
    """3-D points: the same factorization, with the kd ordering cycling through three
    coordinates (block ranks here reach 130 for SE and several hundred for Matern-5/2)."""
    n = 1500
    x, y = I.workload_3d(n, 92)
    th, s2 = [ell, 1.0], 0.01
    sol_d, ld_d = O.dense_solve(x, kern, th, s2, y)
    H = O.Hodlr(x, kern, th, s2, 32, eps, max_rank=1000)
    sol = H.factor_solve(y)
    assert abs(H.logdet() - ld_d) <= tol * abs(ld_d)
    # each level's blocks are off by about eps times their norm (entries <= 1, so <= eps m
    # for an m-point node) and |C^-1| <= 1/sigma^2: |r|/|y| <= eps n kappa / sigma^2
    assert rel_residual(x, kern, th, s2, sol, y) <= eps * n * O.kappa(n, 32) / s2


@pytest.mark.parametrize("n,d,half", [(600, 8, 1.0), (2000, 32, 3.0)])
def test_hodlr_high_dim_vs_dense(n, d, half):
    """High dimension (Sec. 5, the d-dimensional Gaussian tables: C = 2I + exp(-r^2),
    points in [-h, h]^d). d = 8 in a small cube keeps its blocks at full rank; d = 32 in
    [-3, 3]^32 has nearly zero off-diagonal blocks and ranks of a few tens."""
    x = I.uniform_points(n, d, -half, half, 1500 + d)
    y = I.normal(n, 1501 + d)
    th, s2 = [1.0 / np.sqrt(2.0), 1.0], 2.0
    sol_d, ld_d = O.dense_solve(x, "se", th, s2, y)
    H = O.Hodlr(x, "se", th, s2, 32, 1e-12, max_rank=n)
    sol = H.factor_solve(y)
    assert abs(H.logdet() - ld_d) <= 1e-12 * abs(ld_d)
    np.testing.assert_allclose(sol, sol_d, rtol=0, atol=1e-10 * np.abs(sol_d).max())


@pytest.mark.parametrize("kern,d,s2", [("mq", 1, 1.0), ("biharmonic", 1, 2.0), ("mq", 2, 1.0)])
def test_dense_lu_matches_lapack(kern, d, s2):
    """O1 for indefinite C (Sec. 5's multiquadric C = I + K and biharmonic C = 2I + K)
    against LAPACK's LU (numpy slogdet and solve)."""
    n = 700
    x = I.uniform_points(n, d, -3.0, 3.0, 60 + d)
    y = I.normal(n, 61)
    sol, ld, sg = O.dense_lu_solve(x, kern, [1.0, 1.0], s2, y)
    C = dense_C(x, kern, [1.0, 1.0], s2)
    sg_np, ld_np = np.linalg.slogdet(C)
    assert sg == int(sg_np) and abs(ld - ld_np) <= 1e-12 * abs(ld_np)
    ref = np.linalg.solve(C, y)
    np.testing.assert_allclose(sol, ref, rtol=0, atol=1e-10 * np.abs(ref).max())
    assert np.linalg.eigvalsh(C).min() < 0  # the case is really indefinite


@pytest.mark.parametrize("kern,d,s2,eps", [("mq", 1, 1.0, 1e-12), ("biharmonic", 1, 2.0, 1e-12),
                                           ("mq", 2, 1.0, 1e-14), ("biharmonic", 2, 2.0, 1e-12)])
def test_hodlr_indefinite_vs_dense(kern, d, s2, eps):
    """The same factorization on an indefinite C: leaf and node LU determinants may be
    negative, their signs multiply into sign det C (Sec. 4's product of determinants).
    The 2-D multiquadric C has cond ~ 9e5 (smallest |eigenvalue| 0.008), which amplifies
    the compression error (5.7e-10 relative in log |det| at eps = 1e-12, 5.7e-12 at 1e-14);
    it runs at eps = 1e-14."""
    n = 2000
    x = I.uniform_points(n, d, -3.0, 3.0, 70 + d)
    y = I.normal(n, 71)
    sol_d, ld_d, sg_d = O.dense_lu_solve(x, kern, [1.0, 1.0], s2, y)
    H = O.Hodlr(x, kern, [1.0, 1.0], s2, 32, eps, max_rank=1000)
    sol = H.factor_solve(y)
    assert H.logdet_sign() == sg_d
    assert abs(H.logdet() - ld_d) <= 1e-10 * abs(ld_d)
    np.testing.assert_allclose(sol, sol_d, rtol=0, atol=1e-8 * np.abs(sol_d).max())
    with pytest.raises(O.OracleError):
        H.loglik(y)  # not a covariance: no log-likelihood


@pytest.mark.parametrize("kern,theta", [("imq", [0.5, 1.0]), ("rq", [0.3, 1.2, 2.0])])
def test_hodlr_positive_radial_vs_dense(kern, theta):
    n = 2000
    x, y = I.workload_1d(n, 75, lo=-3.0, hi=3.0)
    sol_d, ld_d = O.dense_solve(x, kern, theta, 1.0, y)
    H = O.Hodlr(x, kern, theta, 1.0, 32, 1e-12)
    sol = H.factor_solve(y)
    assert H.logdet_sign() == 1
    assert abs(H.logdet() - ld_d) <= 1e-11 * abs(ld_d)
    np.testing.assert_allclose(sol, sol_d, rtol=0, atol=1e-9 * np.abs(sol_d).max())


# ---------------------------------------------------------------- Chebyshev compression --

@pytest.mark.parametrize("kern,rank", [("exp", 1), ("matern32", 2), ("matern52", 3)])
def test_chebyshev_exact_ranks(kern, rank):
    """On sorted 1-D clusters these kernels are sums of 1 / 2 / 3 separable terms
    (e^{x-y} times 1, (x - y), (x - y)^2), so the recompressed node samples have exactly
    that rank, at every node, whatever q the coefficient test picked."""
    x, _ = I.workload_1d(6000, 51)
    H = O.Hodlr(x, kern, [0.1, 1.0], 0.01, 64, 1e-10, compression="chebyshev")
    assert np.all(H.ranks() == rank)


@pytest.mark.parametrize("kern,ell", [("se", 0.3), ("imq", 0.5), ("rq", 0.4), ("mq", 1.0)])
def test_chebyshev_block_error(kern, ell):
    """||B - U V^T||_F <= C eps ||B||_F for the top block and a deep one (Sec. 3.1's
    interpolation error, C = 100 for the Lebesgue constants and the tail estimate)."""
    x, _ = I.workload_1d(3000, 52, lo=-3.0, hi=3.0)
    eps = 1e-10
    H = O.Hodlr(x, kern, [ell, 1.0], 1.0, 32, eps, max_rank=256, compression="chebyshev")
    xs = x[H.perm(), 0]
    for node in (0, 6):
        U, V = H.node_factors(node)
        (bl, ml), (br, mr) = _node_children(H, node)
        r = np.abs(xs[bl:bl + ml, None] - xs[None, br:br + mr])
        B = O.kernel_values(kern, r.ravel(), ell, 1.0).reshape(r.shape)
        err = np.linalg.norm(B - U @ V.T) / np.linalg.norm(B)
        assert err <= 100 * eps, (node, err)


def _node_children(H, node):
    out = []
    for c in (2 * node + 1, 2 * node + 2):
        b, s = O.ctypes.c_int64(), O.ctypes.c_int64()
        O.lib().oracle_hodlr_node_range(H._h, c, O.ctypes.byref(b), O.ctypes.byref(s))
        out.append((b.value, s.value))
    return out


@pytest.mark.parametrize("kern,ell,s2", [("se", 0.3, 0.01), ("matern52", 0.3, 0.01),
                                         ("imq", 0.5, 1.0), ("mq", 1.0, 1.0)])
def test_chebyshev_hodlr_vs_dense(kern, ell, s2):
    n = 3000
    x, y = I.workload_1d(n, 53, lo=-3.0, hi=3.0)
    x[17] = x[16]  # a duplicated point
    H = O.Hodlr(x, kern, [ell, 1.0], s2, 32, 1e-12, max_rank=256, compression="chebyshev")
    sol = H.factor_solve(y)
    if kern in O.INDEFINITE:
        sol_d, ld_d, sg = O.dense_lu_solve(x, kern, [ell, 1.0], s2, y)
        assert H.logdet_sign() == sg
    else:
        sol_d, ld_d = O.dense_solve(x, kern, [ell, 1.0], s2, y)
    assert abs(H.logdet() - ld_d) <= 1e-11 * abs(ld_d)
    np.testing.assert_allclose(sol, sol_d, rtol=0, atol=1e-8 * np.abs(sol_d).max())


@pytest.mark.parametrize("n", [3, 5, 11, 40])
def test_chebyshev_small_blocks_stored_exactly(n):
    """Leaf size 1: 1 x 2 or 2 x 2 blocks, whose interpolants need more terms than the
    blocks' own rank, are stored exactly; the result is the dense one."""
    x, y = I.workload_1d(n, 65 + n)
    sol_d, ld_d = O.dense_solve(x, "se", [0.5, 1.0], 0.1, y)
    H = O.Hodlr(x, "se", [0.5, 1.0], 0.1, 1, 1e-13, compression="chebyshev")
    sol = H.factor_solve(y)
    assert abs(H.logdet() - ld_d) <= 1e-12 * max(1.0, abs(ld_d))
    np.testing.assert_allclose(sol, sol_d, rtol=0, atol=1e-10 * np.abs(sol_d).max())


def test_chebyshev_reports_nonconvergence():
    """r^2 log r is not smooth where the two clusters meet, and a length scale far below
    the clusters' size needs more than 64 nodes: both report the rank cap status."""
    x, _ = I.workload_1d(2000, 54, lo=-3.0, hi=3.0)
    with pytest.raises(O.OracleError):
        O.Hodlr(x, "biharmonic", [1.0, 1.0], 2.0, 32, 1e-12, compression="chebyshev")
    with pytest.raises(O.OracleError):
        O.Hodlr(x, "se", [0.01, 1.0], 0.01, 32, 1e-12, compression="chebyshev")
    with pytest.raises(O.OracleError):  # 1-D only
        O.Hodlr(I.workload_2d(500, 55)[0], "se", [0.3, 1.0], 0.01, 32, 1e-12,
                compression="chebyshev")


def test_hodlr_matvec_matches_dense():
    n = 800
    x, y = I.workload_1d(n, 95)
    th, s2 = [0.2, 1.0], 0.01
    H = O.Hodlr(x, "matern32", th, s2, 32, 1e-12)
    C = dense_C(x, "matern32", th, s2)
    np.testing.assert_allclose(H.matvec(y), C @ y, rtol=0, atol=1e-12 * np.abs(C @ y).max())


@pytest.mark.parametrize("leaf", [16, 32, 64, 128])
def test_leaf_size_invariance(leaf):
    """Sec. 5.6: the leaf size changes the time, not the result."""
    x, y = I.workload_1d(2048, 97)
    th, s2 = [0.25, 1.0], 0.01
    sol_d, ld_d = O.dense_solve(x, "matern52", th, s2, y)
    H = O.Hodlr(x, "matern52", th, s2, leaf, 1e-13)
    sol = H.factor_solve(y)
    assert abs(H.logdet() - ld_d) <= 1e-11 * abs(ld_d)
    np.testing.assert_allclose(sol, sol_d, rtol=0, atol=1e-9 * np.abs(sol_d).max())


def test_error_decreases_with_eps():
    """The log det error falls with eps and stays below eps relative to |log det|."""
    x, y = I.workload_1d(1024, 99)
    th, s2 = [0.3, 1.0], 0.1
    _, ld_d = O.dense_solve(x, "se", th, s2, y)
    errs = []
    epss = [1e-4, 1e-7, 1e-10]
    for eps in epss:
        H = O.Hodlr(x, "se", th, s2, 32, eps)
        H.factor()
        errs.append(abs(H.logdet() - ld_d))
    assert errs[0] > errs[1] > errs[2]
    for e, eps in zip(errs, epss):
        assert e <= eps * abs(ld_d)


def test_ou_large_vs_hodlr():
    """Exponential kernel at n=2^15: O2 against the closed form (independent)."""
    n = 1 << 15
    x, y = I.workload_1d(n, 1002)
    th, s2 = [0.2, 1.0], 1e-2
    H = O.Hodlr(x, "exp", th, s2, 128, 1e-12)
    sol = H.factor_solve(y)
    p = H.perm()
    sol_c, ld_c = O.ou_closed_form(x[p, 0], th[0], th[1], s2, y[p])
    assert abs(H.logdet() - ld_c) <= 1e-10 * abs(ld_c)
    np.testing.assert_allclose(sol[p], sol_c, rtol=0, atol=1e-8 * np.abs(sol_c).max())


def test_matern32_large_vs_kalman():
    n = 1 << 15
    x, y = I.workload_1d(n, 1003)
    th, s2 = [0.1, 1.0], 1e-2
    H = O.Hodlr(x, "matern32", th, s2, 128, 1e-12)
    sol = H.factor_solve(y)
    p = H.perm()
    ldk, q = O.matern_kalman(x[p, 0], 3, th[0], th[1], s2, y[p])
    assert abs(H.logdet() - ldk) <= 1e-10 * abs(ldk)
    assert abs(y @ sol - q) <= 1e-9 * abs(q)



def test_predict_one_training_point_closed_form():
    """n = 1: mean = k(x*, x1) y1 / (k(0) + s2), var = k(0) - k(x*, x1)^2 / (k(0) + s2)."""
    x = np.array([[0.3]])
    y = np.array([1.7])
    xt = np.array([[0.3], [0.5], [-0.4]])
    th, s2 = [0.2, 1.5], 0.1
    mean, var = O.dense_predict(x, "matern52", th, s2, y, xt)
    k = O.kernel_values("matern52", np.abs(xt[:, 0] - 0.3), 0.2, 1.5)
    np.testing.assert_allclose(mean, k * 1.7 / (1.5 + s2), rtol=1e-14)
    np.testing.assert_allclose(var, 1.5 - k * k / (1.5 + s2), rtol=1e-13, atol=1e-15)


def test_predict_at_training_points_identities():
    """At training point i, C alpha = y gives mean_i = y_i - s2 alpha_i, and
    k_i = C e_i - s2 e_i gives var_i = s2 - s2^2 (C^-1)_ii (both exact identities)."""
    x, y = I.workload_1d(200, 1031)
    s2 = 0.05
    idx = np.arange(0, 200, 17)
    mean, var = O.dense_predict(x, "exp", [0.3, 1.0], s2, y, x[idx])
    alpha, _ = O.dense_solve(x, "exp", [0.3, 1.0], s2, y)
    E = np.zeros((200, len(idx)), order="F")
    E[idx, np.arange(len(idx))] = 1.0
    Cinv_cols, _ = O.dense_solve(x, "exp", [0.3, 1.0], s2, E)
    np.testing.assert_allclose(mean, y[idx] - s2 * alpha[idx], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(var, s2 - s2 * s2 * Cinv_cols[idx, np.arange(len(idx))],
                               rtol=1e-9, atol=1e-13)


def test_predict_matches_scikit_learn():
    """The same posterior from scikit-learn's GP regressor (Matern-3/2, fixed
    hyperparameters, the noise as its diagonal alpha)."""
    gp = pytest.importorskip("sklearn.gaussian_process")
    kern = pytest.importorskip("sklearn.gaussian_process.kernels")
    x, y = I.workload_1d(300, 1032)
    xt = I.uniform_points(25, 1, -1.2, 1.2, 1033)
    th, s2 = [0.15, 1.0], 0.05
    mean, var = O.dense_predict(x, "matern32", th, s2, y, xt)
    k = kern.ConstantKernel(1.0, "fixed") * kern.Matern(length_scale=0.15, nu=1.5,
                                                        length_scale_bounds="fixed")
    reg = gp.GaussianProcessRegressor(kernel=k, alpha=s2, optimizer=None).fit(x, y)
    m2, sd = reg.predict(xt, return_std=True)
    np.testing.assert_allclose(mean, m2, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(var, sd ** 2, rtol=1e-8, atol=1e-10)
