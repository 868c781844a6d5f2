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


def test_struct_layouts_match_header(lib):
    # sizes of the ABI structs on this platform (LP64)
    # ... picard_form and the tail padding to 8 bytes
    assert C.sizeof(rf.rf_solver_params) == 8 * 2 + 4 * 3 + 4 + 8 * 5 + 4 * 3 + 4 + 8 * 2 + 4 * 2 + 4 + 4
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
