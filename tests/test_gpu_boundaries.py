"""Launch-configuration boundaries. A presized context pads every level to the given rank
with zero columns, which leaves every product of the factorization unchanged, so its
log-likelihood must equal the adaptive one. Padding to ranks around each switch and
shared-memory threshold of the level sweep exercises them all on one small problem: the
node step's shared-memory matrix (4 r^2 doubles, opt-in above 40 KB: r = 38, 39, 40), the
fused sweep's limit (r <= 64) and the blocked node step over many CTAs above it (65, 127),
and from r = 128 the level sweep as batched products as well (128, 200)."""
import numpy as np
import pytest

from paper_1403_6015_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_1403_6015_gb300 import build_lib, hodlr
    build_lib.build()
    hodlr.load()
    return hodlr


def rel(a, b):
    return abs(a - b) / abs(b)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("r", [1, 38, 39, 40, 63, 64, 65, 127, 128, 200])
def test_presized_padding_any_rank(H, precision, r):
    x, y = I.workload_1d(1 << 13, 1010)
    th, s2 = [0.3, 1.0], 1e-2
    ref = H.Hodlr(x, "se", th, s2, 64, 1e-12, max_rank=256, precision=precision).loglik(y)
    h = H.Hodlr(x, "se", th, s2, 64, 1e-12, max_rank=256, precision=precision)
    kappa, _ = h.tree()
    # the deepest blocks are 64 x 64: a level's padding beyond its blocks' size is legal
    prof = np.full(kappa, max(r, int(h.ranks().max())), dtype=np.int32)
    h.presize(prof)
    h.rebuild(th, s2)
    got = h.loglik(y)
    assert h.status_flags() == 0
    # padded ranks above 64 run the blocked node step instead of the fused sweep: a
    # different FP64 summation order, carried through the leaf solutions (unit roundoff
    # 2^-53 in the FP64 form, 2^-48 in the double-float leaves of the mixed form; this
    # squared-exponential problem has cond(C) near 1e6; 2.0e-12 seen for the mixed form at
    # r = 65)
    tol_ll = 1e-12 if precision == 0 else 1e-11
    assert rel(got, ref) <= tol_ll, (r, got, ref)
    # and the solve alone with the stored factor (the mixed form's solutions carry its
    # double-float rounding, ~4e-11 of the largest entry here, summed in another order by
    # the unfused sweep than by the fused one)
    sol = h.solve(y)
    sol_ref = H.Hodlr(x, "se", th, s2, 64, 1e-12, max_rank=256, precision=precision).factor_solve(y)
    # above r = 64 the blocked LU and its K-chunked products sum in yet another order: 2.4e-11
    # of the largest entry measured in the FP64 form at r = 128, while every path (fused,
    # blocked) lies 5.3e-10 to 5.5e-10 from the dense solution of this cond ~ 1e6 problem
    tol = (1e-11 if r <= 64 else 1e-10) if precision == 0 else 1e-9
    np.testing.assert_allclose(sol, sol_ref, rtol=0, atol=tol * np.abs(sol_ref).max())


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("max_rank", [2, 256, 257, 341, 512, 8192])
def test_compression_any_max_rank(H, precision, max_rank):
    """The compression's shared memory does not depend on max_rank, but max_rank decides
    which nodes are wide: a rank cap min(m_left, m_right, max_rank) above 256 gives a node
    32-row work items with the sum over earlier cross vectors split over warps (257 and up
    here; 8192 is the largest cap). Ranks here are small, so the result must not depend on
    max_rank. (The smallest cap is 2: the cross takes one step past its last kept term to
    confirm convergence, so even these rank-1 blocks report the cap at max_rank 1.)"""
    x, y = I.workload_1d(1 << 13, 1011)
    th, s2 = [0.2, 1.0], 1e-2
    ref = H.Hodlr(x, "exp", th, s2, 64, 1e-12, precision=precision).loglik(y)
    got = H.Hodlr(x, "exp", th, s2, 64, 1e-12, max_rank=max_rank, precision=precision).loglik(y)
    assert rel(got, ref) <= 1e-13, (max_rank, got, ref)
