"""Autotuner and launch configurations: every configuration computes the same result (up to
the last bits of fixed-order sums), the autotuner picks one of them (leaf CTA size, leaf
kernel, sweep mode and the sweep's tile shape) and can cache it."""
import json

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


@pytest.mark.parametrize("precision", [0, 1])
def test_configurations_agree_and_autotune_picks_one(H, precision):
    """Every launch configuration gives the same log-likelihood: to 1e-13 between CTA
    sizes and sweep modes of one leaf kernel (the order of a few fixed-order sums), to
    1e-12 between the FP32-pipe and the tensor-core leaf kernels of the mixed form (two
    double-float evaluations of the same products, each within ~2^-47 of exact)."""
    n = 1 << 16
    x, y = I.workload_1d(n, 1040)
    h = H.Hodlr(x, "matern32", [0.1, 1.0], 1e-2, 128, 1e-12, precision=precision)
    h.set_tuning(512, 0, 0, 0)
    h.rebuild([0.1, 1.0], 1e-2)
    ref = h.loglik(y)
    cands = ([(512, 0), (1024, 0), (512, 1)] if precision == 1
             else [(256, 0), (512, 0), (1024, 0)])
    for th, kern in cands:
        for mode, tile in ((0, 0), (0, 1), (0, 2), (0, 3), (0, 4), (0, 5), (0, 6), (1, 0)):
            h.set_tuning(th, mode, kern, tile)
            assert h.tuning() == {"leaf_threads": th, "sweep_mode": mode, "leaf_kernel": kern,
                                  "sweep_tile": tile}
            h.rebuild([0.1, 1.0], 1e-2)
            v = h.loglik(y)
            tol = 1e-13 if kern == 0 else 1e-12
            assert abs(v - ref) <= tol * abs(ref), (th, mode, kern, tile, v, ref)
    h.rebuild([0.1, 1.0], 1e-2)
    best = h.autotune(y, reps=2)
    assert (best["leaf_threads"], best["leaf_kernel"]) in cands
    assert best["sweep_mode"] in (0, 1) and best["ms"] > 0
    assert best["sweep_tile"] in range(7)
    assert h.tuning() == {"leaf_threads": best["leaf_threads"], "sweep_mode": best["sweep_mode"],
                          "leaf_kernel": best["leaf_kernel"], "sweep_tile": best["sweep_tile"]}
    v = h.loglik(y)  # the context is compressed and unfactored after the autotuner
    assert abs(v - ref) <= 1e-12 * abs(ref)


def test_tuning_rejects_bad_values(H):
    x, y = I.workload_1d(4096, 1041)
    h = H.Hodlr(x, "exp", [0.2, 1.0], 1e-2, 64, 1e-12, precision=1)
    for th, mode, kern, tile in [(256, 0, 0, 0), (768, 0, 0, 0), (512, 2, 0, 0), (512, 0, 2, 0),
                                 (512, 0, 0, 7), (512, 0, 0, -1)]:  # 256: FP64 only
        with pytest.raises(H.HodlrError):
            h.set_tuning(th, mode, kern, tile)
    h64 = H.Hodlr(x, "exp", [0.2, 1.0], 1e-2, 64, 1e-12, precision=0)
    with pytest.raises(H.HodlrError):
        h64.set_tuning(512, 0, 1)  # the tensor-core leaf kernel is the mixed form's
    with pytest.raises(H.HodlrError):
        h.autotune(y, reps=0)


def test_autotune_cache(H, tmp_path):
    n = 1 << 15
    x, y = I.workload_1d(n, 1042)
    cache = str(tmp_path / "tuning.json")
    h1 = H.Hodlr(x, "matern52", [0.2, 1.0], 1e-2, 128, 1e-12, precision=1)
    r1 = h1.autotune(y, reps=1, cache=cache)
    assert r1["cached"] is False
    table = json.load(open(cache))
    assert len(table) == 1
    h2 = H.Hodlr(x, "matern52", [0.2, 1.0], 1e-2, 128, 1e-12, precision=1)
    r2 = h2.autotune(y, reps=1, cache=cache)
    assert r2["cached"] is True
    assert h2.tuning() == {"leaf_threads": r1["leaf_threads"], "sweep_mode": r1["sweep_mode"],
                           "leaf_kernel": r1["leaf_kernel"], "sweep_tile": r1["sweep_tile"]}
