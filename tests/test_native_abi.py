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


def _header_fields(struct):
    """(type, name) of each member of `typedef struct <struct> { ... } <struct>;`
    in include/nas.h, in order (arrays as 'type[n]')."""
    src = open(os.path.join(ROOT, "include", "nas.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (struct, struct), src, flags=re.S).group(1)
    out = []
    for decl in body.split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        m = re.fullmatch(r"(.+?)\s+(\w+)(?:\[(\w+)\])?", decl)
        typ, name, dim = m.group(1), m.group(2), m.group(3)
        out.append((typ + ("[%s]" % dim if dim else ""), name))
    return out


_CTYPE = {"double": ctypes.c_double, "int": ctypes.c_int, "long long": ctypes.c_longlong}


@pytest.mark.parametrize("struct", ["nas_options", "nas_report"])
def test_binding_structs_match_the_header(libpath, struct):
    """The ctypes structures have the header's members, in its order and
    with its types, so that the library and the binding agree on every
    offset (a member missing on either side shifts all that follow)."""
    from paper_2404_19249_gb300 import nas
    fields = getattr(nas, struct)._fields_
    hdr = _header_fields(struct)
    assert [n for _, n in hdr] == [n for n, _ in fields]
    for (typ, name), (_, ct) in zip(hdr, fields):
        if "[" in typ:
            base, dim = typ[:-1].split("[")
            assert issubclass(ct, ctypes.Array) and ct._type_ is _CTYPE[base], name
        else:
            assert ct is _CTYPE[typ], (name, typ)


def test_trailing_option_defaults(libpath):
    from paper_2404_19249_gb300 import nas
    o = nas.nas_default_options()
    assert (o.smearing, o.inner_adapt, o.bvp_two_level, o.bvp_adapt, o.anderson_restart) == (0.0, 0.0, 0, 0.0, 0.0)
    assert (o.poisson_f32, o.dense_tc, o.density_pairs) == (0, 1, 0)


def test_new_entry_points_check_arguments_before_any_work(libpath):
    """Bad sizes and NULL pointers are refused on the host (no device touched)."""
    from paper_2404_19249_gb300 import nas
    lib, null = nas.lib, None
    p = ctypes.c_void_p(16)      # never dereferenced: every call below fails its argument check first
    assert lib.nas_reconstruct_f64(1, 8, p, p, 0, p, 4, 4, p, p, null) == -1      # N < 1
    assert lib.nas_reconstruct_f64(1, 8, p, p, 65, p, 4, 4, p, p, null) == -1     # tc with N > 64
    assert lib.nas_reconstruct_f64(0, 8, null, p, 4, p, 4, 4, p, p, null) == -1   # NULL icol
    assert lib.nas_gram_sym_f64(1, 8, 65, p, p, p, null) == -1                    # tc with N > 64
    assert lib.nas_gram_sym_f64(0, 8, 91, p, p, p, null) == -1                    # N (N+1)/2 > 4096
    assert lib.nas_gram_sym_f64(0, -1, 4, p, p, p, null) == -1                    # n < 0
    assert lib.nas_dense_precond_f32(0, 8, 0, p, p, p, null) == -1                # k < 1
