"""The C-ABI library builds, loads, and exports every entry point declared in
include/nas.h (no GPU needed; no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "nas.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nas_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2404_19249_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return build.LIB


def test_header_declares_entry_points():
    names = _declared()
    for n in ["nas_create", "nas_set_mesh", "nas_set_system", "nas_init", "nas_step", "nas_solve", "nas_get",
              "nas_apply", "nas_spmm_f64", "nas_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol(libpath):
    from paper_2404_19249_gb300 import nas
    assert sorted(nas.EXPORTS) == _declared()


def test_options_struct_layout(libpath):
    from paper_2404_19249_gb300 import nas
    o = nas.nas_default_options()
    assert o.mu == -1.0 and o.anderson_depth == 5 and abs(o.anderson_beta - 0.7) < 1e-15
    assert o.tol_bvp == 1e-12 and o.max_inner == 50 and o.check_every == 1 and o.hartree == 1
    assert o.eig_dense_max == 1200 and o.timing == 0 and o.eig_device == 1 and o.poisson_two_level == 1
    assert o.eig_adapt == 1e-3 and o.poisson_adaptive == 0 and o.eig_precond == 1
    assert o.poisson_sell == 1 and o.poisson_fused == 0


def test_create_reports_errors_without_crashing(libpath):
    from paper_2404_19249_gb300 import nas
    h = ctypes.c_void_p()
    r = nas.lib.nas_create(ctypes.byref(h), 10 ** 6, None)   # no such device
    assert r == -6 and not h.value
    assert nas.lib.nas_step(None, None) == -1
