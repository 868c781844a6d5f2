"""Host-side argument checking of the C ABI, on the CPU.

rf_mesh_create, rf_ens_create and rf_pcg_solve_noalloc check every argument
before they query the device, so a bad value returns RF_ERR_ARG with its
reason here, on a machine without a GPU, and a good one reaches the device
query (RF_ERR_NO_DEVICE when there is none: no CPU fallback).  No compute call
is made."""
import ctypes as C
import math

import pytest

from paper_1809_10895_gb300 import build as B
from paper_1809_10895_gb300 import rf

NO_GPU = not __import__("torch").cuda.is_available()
needs_no_gpu = pytest.mark.skipif(not NO_GPU, reason="a valid call would create a context on the GPU")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return rf.load()


def _msg(lib):
    return lib.rf_last_error().decode()


def _mesh_create(lib, params=None, mesh=None):
    mesh = mesh if mesh is not None else rf.rf_mesh_desc(4, 3, 5, 1.0, 1.0, 0.5, 0.0, None)
    h = C.c_void_p(1)                       # must be reset to NULL on every error
    st = lib.rf_mesh_create(C.byref(mesh), C.byref(params) if params is not None else None, None, None,
                            C.byref(h))
    return st, _msg(lib), h.value


# (field, bad value, words of the reason)
BAD_PARAMS = [
    ("tol_picard", 0.0, "invalid solver parameters"),
    ("tol_picard", math.nan, "invalid solver parameters"),
    ("tol_cg", -1e-10, "invalid solver parameters"),
    ("cg_max_it", 0, "invalid solver parameters"),
    ("dt0", 0.0, "invalid solver parameters"),
    ("dt_max", -1.0, "invalid solver parameters"),
    ("dt_min", 0.0, "invalid solver parameters"),
    ("f_grow", 0.99, "invalid solver parameters"),
    ("f_shrink", 1.0, "invalid solver parameters"),      # a rejected step must shrink
    ("n_inc", 0, "invalid solver parameters"),
    ("n_small", -1, "invalid solver parameters"),
    ("n_max", 0, "invalid solver parameters"),
    ("eps_chord", -1e-10, "invalid solver parameters"),
    ("tol_inner", 0.0, "invalid solver parameters"),
    ("tol_inner", 1.0, "invalid solver parameters"),
    ("inner_max_it", 0, "invalid solver parameters"),
    ("outer_max_it", 0, "invalid solver parameters"),
    ("precision", 2, "unknown precision"),
    ("precond", 4, "unknown preconditioner"),
    ("picard_form", 2, "unknown Picard linearisation"),
    ("closure_arith", 3, "unknown closure arithmetic"),
    ("face_mean", 2, "unknown interface mean"),
    ("time_scheme", 2, "unknown time scheme"),
    ("time_control", 2, "unknown time control"),
    ("tol_time", math.nan, "tol_time"),
]


# combinations the solver does not run
BAD_COMBOS = [
    (dict(face_mean="harmonic", precision="mixed"), "RF_PREC_FP64"),
    (dict(time_scheme="bdf2"), "modified Picard form under EBATS"),
    (dict(time_scheme="bdf2", picard_form="modified", time_control="richardson"), "under EBATS"),
    (dict(time_control="richardson", tol_time=0.0), "tol_time"),
    (dict(grav=(0.0, math.inf, 1.0)), "gravity"),
]


@pytest.mark.parametrize("kw,why", BAD_COMBOS)
def test_mesh_create_refuses_combinations(lib, kw, why):
    st, msg, h = _mesh_create(lib, rf.default_params(**kw))
    assert st == rf.RF_ERR_ARG and why in msg and h is None


@pytest.mark.parametrize("field,value,why", BAD_PARAMS, ids=[f"{f}={v}" for f, v, _ in BAD_PARAMS])
def test_mesh_create_refuses_bad_params(lib, field, value, why):
    p = rf.default_params()
    setattr(p, field, value)
    st, msg, h = _mesh_create(lib, p)
    assert st == rf.RF_ERR_ARG and why in msg and h is None


@pytest.mark.parametrize("precond", ["mg", "dic", "zline"])
def test_fp32_preconditioners_need_the_mixed_path(lib, precond):
    st, msg, h = _mesh_create(lib, rf.default_params(precision="fp64", precond=precond))
    assert st == rf.RF_ERR_ARG and "RF_PREC_MIXED" in msg and h is None
    st, msg, h = _ens_create(lib, [_instance()], rf.default_params(precision="fp64", precond=precond))
    assert st == rf.RF_ERR_ARG and "RF_PREC_MIXED" in msg and h is None


def test_the_vertical_line_preconditioner_is_the_ensembles(lib):
    st, msg, h = _mesh_create(lib, rf.default_params(precision="mixed", precond="zline"))
    assert st == rf.RF_ERR_ARG and "ensemble" in msg and h is None


@pytest.mark.parametrize("dims,why", [
    ((0, 3, 5, 1.0, 1.0, 0.5), "positive"),
    ((4, 3, -1, 1.0, 1.0, 0.5), "positive"),
    ((4, 3, 5, 0.0, 1.0, 0.5), "positive"),
    ((4, 3, 5, 1.0, math.nan, 0.5), "positive"),
    ((4, 3, 5, 1.0, 1.0, -0.5), "positive"),
    ((2048, 2048, 1024, 1.0, 1.0, 1.0), "too large"),     # 2^32 cells: 32-bit cell indices
])
def test_mesh_create_refuses_bad_meshes(lib, dims, why):
    st, msg, h = _mesh_create(lib, mesh=rf.rf_mesh_desc(*dims, 0.0, None))
    assert st == rf.RF_ERR_ARG and why in msg and h is None


def test_mesh_create_null_arguments(lib):
    h = C.c_void_p(1)
    assert lib.rf_mesh_create(None, None, None, None, C.byref(h)) == rf.RF_ERR_ARG
    assert h.value is None
    mesh = rf.rf_mesh_desc(4, 3, 5, 1.0, 1.0, 0.5, 0.0, None)
    assert lib.rf_mesh_create(C.byref(mesh), None, None, None, None) == rf.RF_ERR_ARG


@needs_no_gpu
@pytest.mark.parametrize("kw", [{}, dict(precision="mixed", precond="mg"), dict(precision="mixed", precond="dic"),
                                dict(picard_form="modified"), dict(f_grow=1.0, n_small=0, eps_chord=0.0),
                                dict(face_mean="harmonic"), dict(time_scheme="bdf2", picard_form="modified"),
                                dict(time_control="richardson"), dict(grav=(0.34, 0.05, 0.94)),
                                dict(closure_arith="double_float"), dict(precision="mixed", closure_arith="fp64")])
def test_valid_params_reach_the_device_query(lib, kw):
    st, msg, h = _mesh_create(lib, rf.default_params(**kw))
    assert st == rf.RF_ERR_NO_DEVICE and "no CPU fallback" in msg and h is None


# ---------------------------------------------------------------- ensemble
def _instance(**kw):
    soil = dict(model=rf.RF_VG, theta_r=0.05, theta_s=0.4, alpha=3.6, n=1.56, Ks=1e-5, S=1e-5)
    soil.update(kw.pop("soil", {}))
    a = dict(nx=2, ny=3, nz=40, dx=0.01, dy=0.01, dz=0.01, h0=-1.0, top_type=rf.BC_TYPES["dirichlet"],
             top_value=0.0, bottom_type=rf.BC_TYPES["free_drainage"], bottom_value=0.0)
    a.update(kw)
    return rf.rf_ens_instance(a["nx"], a["ny"], a["nz"], a["dx"], a["dy"], a["dz"], rf.rf_soil(**soil), a["h0"],
                              a["top_type"], a["top_value"], a["bottom_type"], a["bottom_value"])


def _ens_create(lib, instances, params=None):
    arr = (rf.rf_ens_instance * max(1, len(instances)))(*instances)
    h = C.c_void_p(1)
    st = lib.rf_ens_create(arr, len(instances), C.byref(params) if params is not None else None, None, None,
                           C.byref(h))
    return st, _msg(lib), h.value


@pytest.mark.parametrize("field,value,why", BAD_PARAMS, ids=[f"{f}={v}" for f, v, _ in BAD_PARAMS])
def test_ens_create_refuses_bad_params(lib, field, value, why):
    p = rf.default_params()
    setattr(p, field, value)
    st, msg, h = _ens_create(lib, [_instance()], p)
    assert st == rf.RF_ERR_ARG and why in msg and h is None


@pytest.mark.parametrize("kw,why", [
    (dict(picard_form="modified"), "chord"),
    (dict(precision="mixed", precond="mg"), "Jacobi"),
    (dict(precision="mixed", precond="dic"), "Jacobi"),
    (dict(face_mean="harmonic"), "default scheme"),
    (dict(time_scheme="bdf2", picard_form="modified"), "chord"),
    (dict(time_control="richardson"), "default scheme"),
    (dict(grav=(0.34, 0.05, 0.94)), "default scheme"),
])
def test_ens_create_refuses_forms_it_does_not_run(lib, kw, why):
    st, msg, h = _ens_create(lib, [_instance()], rf.default_params(**kw))
    assert st == rf.RF_ERR_ARG and why in msg and h is None


@pytest.mark.parametrize("kw,why", [
    (dict(nz=0), "bad grid in instance 1"),
    (dict(dx=-0.01), "bad grid in instance 1"),
    (dict(soil=dict(theta_s=0.05)), "bad soil in instance 1"),           # theta_s must exceed theta_r
    (dict(soil=dict(n=1.0)), "bad soil in instance 1"),                   # van Genuchten needs n > 1
    (dict(soil=dict(Ks=0.0)), "bad soil in instance 1"),
    (dict(soil=dict(alpha=0.0)), "bad soil in instance 1"),
    (dict(soil=dict(S=-1e-5)), "bad soil in instance 1"),
    (dict(soil=dict(model=7)), "bad soil in instance 1"),
    (dict(top_type=rf.BC_TYPES["free_drainage"]), "top must be"),
    (dict(bottom_type=rf.BC_TYPES["flux"]), "bottom must be"),
    (dict(nx=2048, ny=2048, nz=600), "too many cells"),
])
def test_ens_create_refuses_bad_instances(lib, kw, why):
    st, msg, h = _ens_create(lib, [_instance(), _instance(**kw)])
    assert st == rf.RF_ERR_ARG and why in msg and h is None


@needs_no_gpu
def test_ens_create_gardner_soil_needs_no_n(lib):
    """n is a van Genuchten parameter only: a Gardner soil with n = 0 passes the
    checks and reaches the device query."""
    st, msg, h = _ens_create(lib, [_instance(soil=dict(model=rf.RF_GARDNER, n=0.0))])
    assert st == rf.RF_ERR_NO_DEVICE and h is None, msg


def test_ens_create_needs_an_instance(lib):
    st, msg, h = _ens_create(lib, [])
    assert st == rf.RF_ERR_ARG and "at least one instance" in msg and h is None


@needs_no_gpu
@pytest.mark.parametrize("precond", ["jacobi", "zline"])
def test_valid_ensemble_reaches_the_device_query(lib, precond):
    st, msg, h = _ens_create(lib, [_instance(), _instance(nx=16, ny=16, nz=400)],
                             rf.default_params(precision="mixed", precond=precond))
    assert st == rf.RF_ERR_NO_DEVICE and "no CPU fallback" in msg and h is None


# ------------------------------------------------- allocation-free solve
FAKE = C.c_void_p(4096)                    # never dereferenced: every case below fails its checks first


@pytest.mark.parametrize("args,why", [
    ((0, 4, 4, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, 1e-10, 100), "invalid argument"),
    ((4, 4, 4, None, FAKE, FAKE, FAKE, FAKE, FAKE, 1e-10, 100), "invalid argument"),
    ((4, 4, 4, FAKE, FAKE, FAKE, FAKE, FAKE, None, 1e-10, 100), "invalid argument"),
    ((4, 4, 4, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, 0.0, 100), "invalid argument"),
    ((4, 4, 4, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, math.nan, 100), "invalid argument"),
    ((4, 4, 4, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, 1e-10, 0), "invalid argument"),
    ((64, 64, 17, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, 1e-10, 100), "RF_NOALLOC_MAX_CELLS"),
])
def test_noalloc_solve_refuses_bad_arguments(lib, args, why):
    it = C.c_int(-1)
    st = lib.rf_pcg_solve_noalloc(*args, None, C.byref(it))
    assert st == rf.RF_ERR_ARG and why in _msg(lib)
    assert 64 * 64 * 17 > rf.NOALLOC_MAX_CELLS >= 64 * 64 * 16
