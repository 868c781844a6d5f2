"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports
every function include/rf.h declares, and refuses to run without a GPU (no
CPU fallback).  No compute call is made here."""
import ctypes as C
import os

import pytest

from paper_1809_10895_gb300 import build as B
from paper_1809_10895_gb300 import rf

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "rf.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return rf.load()


def test_every_declared_symbol_is_exported(lib):
    names = rf.header_function_names(HEADER)
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
        assert n in rf.SIGNATURES, f"binding lacks {n}"


def test_default_params_match_documented_defaults(lib):
    p = rf.default_params()
    assert (p.tol_picard, p.tol_cg, p.cg_max_it) == (1e-6, 1e-10, 10000)
    assert (p.dt0, p.dt_max, p.dt_min, p.f_grow, p.f_shrink) == (1.0, 600.0, 1e-3, 1.3, 1.3)
    assert (p.n_inc, p.n_small, p.n_max) == (10, 3, 8)
    assert p.picard_form == rf.PICARD_FORM["chord"]
    assert (p.closure_arith, p.face_mean, p.time_scheme, p.time_control) == (0, 0, 0, 0)
    assert p.tol_time == 1e-3 and tuple(p.grav) == (0.0, 0.0, 1.0)


def test_struct_layouts_match_header(lib):
    # sizes of the ABI structs on this platform (LP64)
    # ... picard_form, closure_arith, face_mean, time_scheme, time_control
    # (+4 padding), tol_time, grav[3]
    assert C.sizeof(rf.rf_solver_params) == 8 * 2 + 4 * 3 + 4 + 8 * 5 + 4 * 3 + 4 + 8 * 2 + 4 * 2 + 4 * 5 + 4 + 8 + 8 * 3
    # rf_ens_stats: t, dt_nom; 4 counters; status (+4); cells; 5 balances; busy_s; ctas (+4)
    assert C.sizeof(rf.rf_ens_stats) == 8 * 2 + 8 * 4 + 4 + 4 + 8 + 8 * 5 + 8 + 4 + 4
    assert C.sizeof(rf.rf_step_info) == 8 * 2 + 4 * 3 + 4 + 8
    assert C.sizeof(rf.rf_mesh_desc) == 4 * 3 + 4 + 8 * 4 + 8


@pytest.mark.skipif(__import__("torch").cuda.is_available(), reason="needs a machine without a GPU")
def test_no_gpu_means_no_device_error(lib):
    desc = rf.rf_mesh_desc(2, 2, 2, 1.0, 1.0, 1.0, 0.0, None)
    h = C.c_void_p()
    st = lib.rf_mesh_create(C.byref(desc), None, None, None, C.byref(h))
    assert st == rf.RF_ERR_NO_DEVICE
    assert b"no CPU fallback" in lib.rf_last_error() or b"no CUDA device" in lib.rf_last_error()
    assert not h.value


def _prototypes(header):
    """(return type, name, [parameter types]) of every function declared in
    the header, comments removed."""
    import re
    txt = re.sub(r"/\*.*?\*/", "", open(header).read(), flags=re.S)
    txt = re.sub(r"#[^\n]*", "", txt)
    out = []
    for m in re.finditer(r"([A-Za-z_][A-Za-z_0-9 \*]*?)\b(rf_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", txt):
        ret, name, params = m.group(1).split("\n")[-1].strip(), m.group(2), m.group(3)
        plist = [p.strip() for p in params.replace("\n", " ").split(",")]
        plist = [] if plist == ["void"] or plist == [""] else plist
        out.append((ret, name, plist))
    return out


def _header_kind(decl):
    """The ABI class of a C declaration (parameter with or without a name)."""
    if "*" in decl:
        return "ptr"
    words = decl.replace("const", "").split()
    if words[:2] == ["unsigned", "long"]:
        return "u64"
    if words[:2] == ["long", "long"]:
        return "i64"
    if words[0] == "double":
        return "f64"
    if words[0] == "float":
        return "f32"
    if words[0] == "void":
        return "void"
    if words[0] in ("int", "rf_status", "rf_face", "rf_bc_type", "rf_precision", "rf_precond", "rf_picard_form"):
        return "i32"
    raise AssertionError(f"unclassified C type in {decl!r}")


def _ctypes_kind(t):
    if t is None:
        return "void"
    if t in (C.c_void_p, C.c_char_p) or (isinstance(t, type) and issubclass(t, C._Pointer)):
        return "ptr"
    return {C.c_int: "i32", C.c_double: "f64", C.c_float: "f32", C.c_longlong: "i64", C.c_ulonglong: "u64"}[t]


def test_binding_signatures_match_header_prototypes():
    protos = _prototypes(HEADER)
    names = [n for _, n, _ in protos]
    assert sorted(names) == rf.header_function_names(HEADER)
    for ret, name, params in protos:
        restype, argtypes = rf.SIGNATURES[name]
        assert _ctypes_kind(restype) == _header_kind(ret), name
        assert len(argtypes) == len(params), (name, len(argtypes), params)
        for i, (a, p) in enumerate(zip(argtypes, params)):
            assert _ctypes_kind(a) == _header_kind(p), (name, i, p)


def test_binding_constants_match_header():
    import re
    txt = open(HEADER).read()
    consts = dict(re.findall(r"#define\s+(RF_[A-Z_]+)\s+(\d+)", txt))
    assert int(consts["RF_NOALLOC_MAX_CELLS"]) == rf.NOALLOC_MAX_CELLS
    assert int(consts["RF_NN_PARAMS"]) == rf.NN_PARAMS
