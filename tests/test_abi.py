"""CPU checks of the boundary: the library builds, loads, and exports every entry point the
header declares (no compute calls: there may be no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "hodlr.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hodlr_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1403_6015_gb300 import build_lib
    return ctypes.CDLL(build_lib.build())


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ["hodlr_build", "hodlr_factor", "hodlr_solve", "hodlr_logdet", "hodlr_loglik",
              "hodlr_destroy", "hodlr_last_error"]:
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_names_match_abi():
    from paper_1403_6015_gb300 import hodlr
    for s in declared_symbols():
        assert hasattr(hodlr, s), s


def test_status_strings(lib):
    lib.hodlr_status_string.restype = ctypes.c_char_p
    assert lib.hodlr_status_string(0) == b"OK"
    assert lib.hodlr_status_string(3) == b"ENOTSPD"


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1403_6015_gb300 import hodlr
    monkeypatch.setattr(hodlr, "_lib", None)
    monkeypatch.setattr(hodlr, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        hodlr.load()


def test_product_path_does_not_touch_oracle():
    """The package never imports, links, loads or runs anything under oracle/."""
    pat = re.compile(r"import\s+oracle|from\s+oracle|liboracle|hodlr_oracle|oracle[/\\]|"
                     r"oracle_[a-z]+\(")
    pkg = os.path.join(ROOT, "paper_1403_6015_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not pat.search(src), os.path.join(dirpath, f)


def test_build_rejects_bad_options():
    """Refinement and rank-cap checks happen before any device work (no GPU needed)."""
    import numpy as np

    from paper_1403_6015_gb300 import hodlr
    x = np.linspace(0, 1, 64)
    for maxit, tol in [(-1, 1e-10), (2, 0.0), (2, float("nan"))]:
        o = hodlr.hodlr_default_opts()
        o.refine_maxit = maxit
        o.refine_tol = tol
        st, ctx = hodlr.hodlr_build(x, 64, 1, 0, [0.2, 1.0], 0.01, 16, 1e-12, o)
        assert st == hodlr.HODLR_EINVAL and not ctx
    for mr in [0, 8193]:
        o = hodlr.hodlr_default_opts()
        o.max_rank = mr
        st, ctx = hodlr.hodlr_build(x, 64, 1, 0, [0.2, 1.0], 0.01, 16, 1e-12, o)
        assert st == hodlr.HODLR_EINVAL and not ctx
    assert hodlr.hodlr_default_opts().max_rank == 64
    # the rational quadratic needs alpha > 0; the indefinite kernels (multiquadric,
    # biharmonic) need the FP64 form; kernel codes end at 7; d at most 64
    assert hodlr.hodlr_default_opts().rq_alpha == 1.0
    for a in [0.0, -1.0, float("nan"), float("inf")]:
        o = hodlr.hodlr_default_opts()
        o.rq_alpha = a
        st, ctx = hodlr.hodlr_build(x, 64, 1, hodlr.KERNELS["rq"], [0.2, 1.0], 0.01, 16, 1e-12, o)
        assert st == hodlr.HODLR_EINVAL and not ctx
    for kern in hodlr.INDEFINITE:
        o = hodlr.hodlr_default_opts()
        o.precision = 1
        st, ctx = hodlr.hodlr_build(x, 64, 1, hodlr.KERNELS[kern], [0.2, 1.0], 0.01, 16, 1e-12, o)
        assert st == hodlr.HODLR_EINVAL and not ctx
    st, ctx = hodlr.hodlr_build(x, 64, 1, 8, [0.2, 1.0], 0.01, 16, 1e-12, None)
    assert st == hodlr.HODLR_EINVAL and not ctx
    # Chebyshev compression: codes 0/1 only, points in 1-D only
    for comp, xx, d in [(2, x, 1), (-1, x, 1), (1, np.zeros((64, 2)), 2)]:
        o = hodlr.hodlr_default_opts()
        o.compression = comp
        st, ctx = hodlr.hodlr_build(xx, 64, d, 1, [0.2, 1.0], 0.01, 16, 1e-12, o)
        assert st == hodlr.HODLR_EINVAL and not ctx
    assert hodlr.hodlr_default_opts().compression == 0
    x65 = np.zeros((2, 65))
    st, ctx = hodlr.hodlr_build(x65, 2, 65, 0, [0.2, 1.0], 0.01, 16, 1e-12, None)
    assert st == hodlr.HODLR_EINVAL and not ctx
