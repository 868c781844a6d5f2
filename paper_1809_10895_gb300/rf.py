"""Thin ctypes binding of the C ABI in ``include/rf.h`` (``_build/librf.so``).

Argument marshalling only: every step of the numerical path runs in the CUDA
kernels behind the ABI.  PyTorch supplies device memory (through the ABI's
allocator callback, so the library's buffers come from torch's caching
allocator) and the CUDA stream.  There is no CPU fallback: loading fails
loudly when the library is missing, and creating a solver fails without an
sm_103 GPU.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librf.so")

RF_OK, RF_ERR_ARG, RF_ERR_NO_DEVICE, RF_ERR_CUDA, RF_ERR_NOMEM, RF_ERR_STATE, RF_ERR_PICARD, \
    RF_ERR_DT_MIN, RF_ERR_CG, RF_ERR_DEVICE_TIMEOUT = range(10)
STATUS_NAMES = ("RF_OK", "RF_ERR_ARG", "RF_ERR_NO_DEVICE", "RF_ERR_CUDA", "RF_ERR_NOMEM", "RF_ERR_STATE",
                "RF_ERR_PICARD", "RF_ERR_DT_MIN", "RF_ERR_CG", "RF_ERR_DEVICE_TIMEOUT")
RF_VG, RF_GARDNER, RF_BROOKS_COREY = 0, 1, 2
FACES = {"xmin": 0, "xmax": 1, "ymin": 2, "ymax": 3, "zmin": 4, "zmax": 5}
BC_TYPES = {"zero_flux": 0, "dirichlet": 1, "flux": 2, "free_drainage": 3, "seepage": 4}
MODELS = {"vg": RF_VG, "gardner": RF_GARDNER, "brooks_corey": RF_BROOKS_COREY}
PRECISION = {"fp64": 0, "mixed": 1}
PRECOND = {"jacobi": 0, "mg": 1, "dic": 2, "zline": 3}
PICARD_FORM = {"chord": 0, "modified": 1}
CLOSURE_ARITH = {"auto": 0, "fp64": 1, "double_float": 2}
FACE_MEAN = {"arithmetic": 0, "harmonic": 1}
TIME_SCHEME = {"backward_euler": 0, "bdf2": 1}
TIME_CONTROL = {"ebats": 0, "richardson": 1}
_ENUM_PARAMS = {"precision": PRECISION, "precond": PRECOND, "picard_form": PICARD_FORM,
                "closure_arith": CLOSURE_ARITH, "face_mean": FACE_MEAN, "time_scheme": TIME_SCHEME,
                "time_control": TIME_CONTROL}


class rf_solver_params(C.Structure):
    _fields_ = [("tol_picard", C.c_double), ("tol_cg", C.c_double), ("cg_max_it", C.c_int),
                ("precond", C.c_int), ("precision", C.c_int), ("dt0", C.c_double), ("dt_max", C.c_double),
                ("dt_min", C.c_double), ("f_grow", C.c_double), ("f_shrink", C.c_double), ("n_inc", C.c_int),
                ("n_small", C.c_int), ("n_max", C.c_int), ("eps_chord", C.c_double), ("tol_inner", C.c_double),
                ("inner_max_it", C.c_int), ("outer_max_it", C.c_int), ("picard_form", C.c_int),
                ("closure_arith", C.c_int), ("face_mean", C.c_int), ("time_scheme", C.c_int),
                ("time_control", C.c_int), ("tol_time", C.c_double), ("grav", C.c_double * 3)]


class rf_mesh_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double), ("dy", C.c_double),
                ("dz", C.c_double), ("z_bottom", C.c_double), ("active", C.POINTER(C.c_uint8))]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class rf_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class rf_soil(C.Structure):
    _fields_ = [("model", C.c_int), ("theta_r", C.c_double), ("theta_s", C.c_double), ("alpha", C.c_double),
                ("n", C.c_double), ("Ks", C.c_double), ("S", C.c_double)]


class rf_state_meta(C.Structure):
    _fields_ = [("t", C.c_double), ("dt_nom", C.c_double), ("easy", C.c_int), ("n_active", C.c_int),
                ("steps", C.c_longlong)]


class rf_step_info(C.Structure):
    _fields_ = [("dt", C.c_double), ("t", C.c_double), ("picard_iters", C.c_int), ("cg_iters", C.c_int),
                ("rejected", C.c_int), ("max_dh", C.c_double)]


class rf_run_stats(C.Structure):
    _fields_ = [("steps", C.c_longlong), ("picard_iters", C.c_longlong), ("cg_iters", C.c_longlong),
                ("rejected", C.c_longlong)]


class rf_mass_balance_t(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("storage0", "storage", "inflow_cum", "outflow_cum", "closure_abs",
                                          "closure_rel", "nonlinear_defect_cum")]


class rf_ens_instance(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double), ("dy", C.c_double),
                ("dz", C.c_double), ("soil", rf_soil), ("h0", C.c_double), ("top_type", C.c_int),
                ("top_value", C.c_double), ("bottom_type", C.c_int), ("bottom_value", C.c_double)]


class rf_ens_stats(C.Structure):
    _fields_ = [("t", C.c_double), ("dt_nom", C.c_double), ("steps", C.c_longlong), ("picard_iters", C.c_longlong),
                ("cg_iters", C.c_longlong), ("rejected", C.c_longlong), ("status", C.c_int), ("cells", C.c_longlong),
                ("storage0", C.c_double), ("inflow_cum", C.c_double), ("outflow_cum", C.c_double),
                ("closure_abs", C.c_double), ("nonlinear_defect_cum", C.c_double), ("busy_s", C.c_double),
                ("ctas", C.c_int)]


class rf_ws_scales(C.Structure):
    _fields_ = [("h_scale", C.c_double), ("lnK_mean", C.c_double), ("lnK_std", C.c_double), ("q_scale", C.c_double),
                ("t_scale", C.c_double), ("out_scale", C.c_double)]


class rf_adam(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float)]


class rf_ws_stats(C.Structure):
    _fields_ = [("guesses", C.c_longlong), ("fallbacks", C.c_longlong)]


# name -> (restype, argtypes): the functions declared in include/rf.h
_VP, _DP, _U8P = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_uint8)
SIGNATURES = {
    "rf_default_params": (None, [C.POINTER(rf_solver_params)]),
    "rf_last_error": (C.c_char_p, []),
    "rf_mesh_create": (C.c_int, [C.POINTER(rf_mesh_desc), C.POINTER(rf_solver_params), _VP,
                                 C.POINTER(rf_allocator), C.POINTER(_VP)]),
    "rf_destroy": (None, [_VP]),
    "rf_set_params": (C.c_int, [_VP, C.POINTER(rf_solver_params)]),
    "rf_soil_set": (C.c_int, [_VP, C.POINTER(rf_soil), C.c_int, _U8P, _DP]),
    "rf_bc_set": (C.c_int, [_VP, C.c_int, C.c_int, _DP, _DP, C.c_int]),
    "rf_state_set": (C.c_int, [_VP, _DP, C.c_double]),
    "rf_state_set_device": (C.c_int, [_VP, _VP, C.c_double]),
    "rf_state_get": (C.c_int, [_VP, _DP, C.POINTER(rf_state_meta)]),
    "rf_state_get_device": (C.c_int, [_VP, _VP]),
    "rf_state_meta_set": (C.c_int, [_VP, C.POINTER(rf_state_meta), _DP]),
    "rf_step": (C.c_int, [_VP, C.POINTER(rf_step_info)]),
    "rf_run": (C.c_int, [_VP, C.c_double, C.POINTER(rf_run_stats), C.POINTER(rf_step_info), C.c_int]),
    "rf_mass_balance": (C.c_int, [_VP, C.POINTER(rf_mass_balance_t)]),
    "rf_assemble": (C.c_int, [_VP, _VP, _VP, C.c_double, C.c_double, _VP, _VP, _VP, _VP, _VP]),
    "rf_apply": (C.c_int, [_VP, _VP, _VP]),
    "rf_solve": (C.c_int, [_VP, _VP, C.POINTER(C.c_int)]),
    "rf_apply_inner": (C.c_int, [_VP, _VP, _VP, C.c_float, _VP, _VP, _DP]),
    "rf_set_wait_limit": (C.c_int, [_VP, C.c_int]),
    "rf_launch_count": (C.c_ulonglong, [_VP]),
    "rf_profile_kernel": (C.c_int, [_VP, C.c_int, C.c_int, _DP, _DP]),
    "rf_launch_counts": (C.c_int, [_VP, C.POINTER(C.c_ulonglong), C.c_int]),
    "rf_ens_create": (C.c_int, [C.POINTER(rf_ens_instance), C.c_int, C.POINTER(rf_solver_params), _VP,
                                C.POINTER(rf_allocator), C.POINTER(_VP)]),
    "rf_ens_destroy": (None, [_VP]),
    "rf_ens_set_tiling": (C.c_int, [_VP, C.c_int, C.c_int]),
    "rf_ens_set_schedule": (C.c_int, [_VP, C.POINTER(C.c_int), C.c_int]),
    "rf_ens_run": (C.c_int, [_VP, C.c_double]),
    "rf_ens_get": (C.c_int, [_VP, C.c_int, _DP, C.POINTER(rf_ens_stats)]),
    "rf_ens_reset": (C.c_int, [_VP]),
    "rf_ens_tune": (C.c_int, [_VP, C.c_double, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), _DP]),
    "rf_ens_model_makespan": (C.c_int, [_DP, _DP, C.POINTER(C.c_int), C.c_int, C.c_int, C.c_int, C.c_int, _DP]),
    "rf_pcg_solve_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, _VP, _VP, _VP, _VP, _VP, _VP, C.c_double,
                                       C.c_int, _VP, C.POINTER(C.c_int)]),
    "rf_nn_create": (C.c_int, [_VP, C.POINTER(rf_allocator), C.POINTER(_VP)]),
    "rf_nn_destroy": (None, [_VP]),
    "rf_nn_set_params": (C.c_int, [_VP, _VP, C.c_longlong]),
    "rf_nn_get_params": (C.c_int, [_VP, _VP, C.c_longlong]),
    "rf_nn_forward": (C.c_int, [_VP, _VP, C.c_int, C.c_int, C.c_int, C.c_int, _VP]),
    "rf_nn_loss_grad": (C.c_int, [_VP, _VP, _VP, _VP, C.c_int, C.c_int, C.c_int, C.c_int,
                                  C.POINTER(C.c_float), _VP]),
    "rf_nn_train_step": (C.c_int, [_VP, _VP, _VP, _VP, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(rf_adam),
                                   C.POINTER(C.c_float)]),
    "rf_nn_launch_count": (C.c_longlong, [_VP]),
    "rf_nn_set_trace": (C.c_int, [_VP, C.c_int]),
    "rf_nn_trace_get": (C.c_int, [_VP, C.c_int, C.c_int, _VP, C.c_longlong]),
    "rf_ws_features": (C.c_int, [_VP, C.POINTER(rf_ws_scales), _VP, C.c_double, C.c_double, _VP]),
    "rf_ws_target": (C.c_int, [_VP, C.POINTER(rf_ws_scales), _VP, C.c_double, _VP, _VP]),
    "rf_ws_attach": (C.c_int, [_VP, _VP, C.POINTER(rf_ws_scales)]),
    "rf_ws_get_stats": (C.c_int, [_VP, C.POINTER(rf_ws_stats)]),
}
NOALLOC_MAX_CELLS = 65536
NN_PARAMS = 225793
NN_LAYERS = 10
COUNTER_KINDS = ("closure", "closure_picard", "assemble", "cg64_init", "cg64_spmv", "cg64_update", "apply64",
                 "mixed_start", "resid64", "cg32_spmv", "cg32_update", "add_correction", "mass_balance",
                 "storage", "accept")
KERNEL_KINDS = {"closure": 0, "assemble": 1, "cg64_spmv": 2, "cg64_update": 3, "resid64": 4, "cg32_spmv": 5,
                "cg32_update": 6}

_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build()); "
                               "there is no CPU fallback")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class RFError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load().rf_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


def _check(st: int, where: str):
    if st != RF_OK:
        raise RFError(st, where)


def default_params(**kw) -> rf_solver_params:
    p = rf_solver_params()
    load().rf_default_params(C.byref(p))
    _set_params(p, kw)
    return p


def _set_params(p: rf_solver_params, kw: dict):
    """Parameter names as in rf_solver_params; enumerations may be given by
    name; grav_x / grav_y / grav_z set the components of grav."""
    for k, v in kw.items():
        if k in _ENUM_PARAMS and isinstance(v, str):
            v = _ENUM_PARAMS[k][v]
        if k in ("grav_x", "grav_y", "grav_z"):
            p.grav["xyz".index(k[-1])] = float(v)
        elif k == "grav":
            for i in range(3):
                p.grav[i] = float(v[i])
        elif k in dict(rf_solver_params._fields_):
            setattr(p, k, v)
        else:
            raise KeyError(f"unknown solver parameter {k!r}")


def _dptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(_DP)


class TorchAllocator:
    """Device memory for the library from torch's caching allocator."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device
        self.blocks = {}
        self._alloc = ALLOC_FN(self._do_alloc)
        self._free = FREE_FN(self._do_free)
        self.struct = rf_allocator(self._alloc, self._free, None)

    def _do_alloc(self, nbytes, user):
        t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        ptr = t.data_ptr()
        self.blocks[ptr] = t
        return ptr

    def _do_free(self, ptr, user):
        self.blocks.pop(ptr, None)


@dataclass
class StepInfo:
    dt: float
    t: float
    picard: int
    cg: int
    rejected: int
    max_dh: float

    @staticmethod
    def of(s: rf_step_info) -> "StepInfo":
        return StepInfo(s.dt, s.t, s.picard_iters, s.cg_iters, s.rejected, s.max_dh)


class Solver:
    """One solver context on the current CUDA device and torch stream."""

    def __init__(self, nx, ny, nz, dx, dy, dz, z_bottom=0.0, active=None, params=None, stream=None,
                 use_torch_allocator=True):
        import torch
        L = load()
        self.shape = (nx, ny, nz)
        self.N = nx * ny * nz
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._active = None if active is None else np.ascontiguousarray(active, dtype=np.uint8).ravel()
        desc = rf_mesh_desc(nx, ny, nz, dx, dy, dz, z_bottom,
                            None if self._active is None else self._active.ctypes.data_as(_U8P))
        self.params = params if params is not None else default_params()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._allocator = TorchAllocator(self.device) if use_torch_allocator else None
        h = _VP()
        _check(L.rf_mesh_create(C.byref(desc), C.byref(self.params), C.c_void_p(self.stream.cuda_stream),
                                C.byref(self._allocator.struct) if self._allocator else None, C.byref(h)),
               "rf_mesh_create")
        self.ctx = h

    def close(self):
        if getattr(self, "ctx", None):
            load().rf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- set-up
    @classmethod
    def from_case(cls, case, **param_overrides) -> "Solver":
        """Build a solver from a workloads.Case (mesh, soils, BCs, params, state)."""
        p = dict(case.params)
        p["grav"] = tuple(getattr(case, "gravity", (0.0, 0.0, 1.0)))
        p.update(param_overrides)
        s = cls(case.nx, case.ny, case.nz, case.dx, case.dy, case.dz, case.z_bottom, case.active,
                params=default_params(**p))
        s.set_soils(case.soils, case.zone_of_cell, case.Ks_cell)
        for bc in case.bcs:
            s.set_bc(bc.face, bc.type, bc.t, bc.v)
        s.set_state(case.h0, case.t0)
        return s

    def set_params(self, **kw):
        p = self.params
        _set_params(p, kw)
        _check(load().rf_set_params(self.ctx, C.byref(p)), "rf_set_params")

    def set_soils(self, soils, zone_of_cell=None, Ks_cell=None):
        arr = (rf_soil * len(soils))()
        for i, s in enumerate(soils):
            arr[i] = rf_soil(MODELS[s.get("model", "vg")], s["theta_r"], s["theta_s"], s["alpha"],
                             s.get("n", 2.0), s["Ks"], s.get("S", 1e-5))
        z = None if zone_of_cell is None else np.ascontiguousarray(zone_of_cell, dtype=np.uint8).ravel()
        k = None if Ks_cell is None else np.ascontiguousarray(Ks_cell, dtype=np.float64).ravel()
        _check(load().rf_soil_set(self.ctx, arr, len(soils), None if z is None else z.ctypes.data_as(_U8P),
                                  _dptr(k)), "rf_soil_set")

    def set_bc(self, face, type_, t=None, v=None):
        if v is None:
            _check(load().rf_bc_set(self.ctx, FACES[face], BC_TYPES[type_], None, None, 0), "rf_bc_set")
            return
        v = np.ascontiguousarray(np.atleast_1d(v), dtype=np.float64)
        t = (np.zeros(len(v)) if t is None else np.ascontiguousarray(np.atleast_1d(t), dtype=np.float64))
        _check(load().rf_bc_set(self.ctx, FACES[face], BC_TYPES[type_], _dptr(t), _dptr(v), len(v)), "rf_bc_set")

    def set_state(self, h, t=0.0):
        h = np.ascontiguousarray(h, dtype=np.float64).ravel()
        _check(load().rf_state_set(self.ctx, _dptr(h), float(t)), "rf_state_set")

    def set_state_device(self, h_dev, t=0.0):
        _check(load().rf_state_set_device(self.ctx, C.c_void_p(h_dev.data_ptr()), float(t)), "rf_state_set_device")

    # -- stepping
    def step(self) -> StepInfo:
        info = rf_step_info()
        _check(load().rf_step(self.ctx, C.byref(info)), "rf_step")
        return StepInfo.of(info)

    def run(self, t_end, log_cap=1_000_000):
        stats = rf_run_stats()
        log = (rf_step_info * max(log_cap, 1))()
        st = load().rf_run(self.ctx, float(t_end), C.byref(stats), log, log_cap)
        steps = [StepInfo.of(log[i]) for i in range(min(stats.steps, log_cap))]
        _check(st, "rf_run")
        return steps

    def get_state(self, out=None):
        """(h, meta); h is written into out (a contiguous float64 array of N
        cells, e.g. a view of pinned memory, so the copy runs at full rate)
        when given, else into a new array."""
        if out is None:
            h = np.empty(self.N)
        else:
            h = out
            if not (isinstance(h, np.ndarray) and h.dtype == np.float64 and h.size == self.N and h.flags.c_contiguous):
                raise ValueError("get_state: out must be a contiguous float64 array of N cells")
        meta = rf_state_meta()
        _check(load().rf_state_get(self.ctx, _dptr(h), C.byref(meta)), "rf_state_get")
        return h, dict(t=meta.t, dt_nom=meta.dt_nom, easy=meta.easy, n_active=meta.n_active, steps=meta.steps)

    def get_state_device(self, out):
        _check(load().rf_state_get_device(self.ctx, C.c_void_p(out.data_ptr())), "rf_state_get_device")
        return out

    def set_meta(self, meta: dict, mass7=None):
        m = rf_state_meta(meta["t"], meta["dt_nom"], meta["easy"], meta.get("n_active", 0), meta.get("steps", 0))
        arr = None if mass7 is None else np.ascontiguousarray(mass7, dtype=np.float64)
        _check(load().rf_state_meta_set(self.ctx, C.byref(m), _dptr(arr)), "rf_state_meta_set")

    def mass_balance(self) -> dict:
        mb = rf_mass_balance_t()
        _check(load().rf_mass_balance(self.ctx, C.byref(mb)), "rf_mass_balance")
        return {k: getattr(mb, k) for k, _ in rf_mass_balance_t._fields_}

    def launch_count(self) -> int:
        return int(load().rf_launch_count(self.ctx))

    def launch_counts(self) -> dict:
        """{kind: (launches, launches that did work)} from the device counters."""
        buf = (C.c_ulonglong * (2 * len(COUNTER_KINDS)))()
        n = load().rf_launch_counts(self.ctx, buf, len(buf))
        return {k: (int(buf[2 * i]), int(buf[2 * i + 1])) for i, k in enumerate(COUNTER_KINDS) if 2 * i + 1 < n}

    def profile_kernel(self, kind: str, reps: int = 50):
        """(mean ms per launch, algorithmic bytes per launch) of one kernel."""
        ms, by = C.c_double(0), C.c_double(0)
        _check(load().rf_profile_kernel(self.ctx, KERNEL_KINDS[kind], reps, C.byref(ms), C.byref(by)),
               "rf_profile_kernel")
        return ms.value, by.value

    # -- kernel level (torch CUDA float64 tensors of N elements)
    def assemble(self, hk, hn, dt, t=0.0, K=None, theta=None, c=None, b=None, diag=None):
        ptr = lambda a: None if a is None else C.c_void_p(a.data_ptr())
        _check(load().rf_assemble(self.ctx, ptr(hk), ptr(hn), float(dt), float(t), ptr(K), ptr(theta), ptr(c),
                                  ptr(b), ptr(diag)), "rf_assemble")

    def apply(self, x, y):
        _check(load().rf_apply(self.ctx, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr())), "rf_apply")

    def solve(self, x) -> int:
        it = C.c_int(0)
        _check(load().rf_solve(self.ctx, C.c_void_p(x.data_ptr()), C.byref(it)), "rf_solve")
        return it.value

    def apply_inner(self, z, p_out, q_out, pold=None, beta=0.0) -> float:
        """The FP32 inner-solve stencil step on the last assembled system
        (torch CUDA float32 tensors of N elements): p = z + beta pold,
        q = A32 p; returns p . q."""
        import torch
        for name, a in (("z", z), ("p_out", p_out), ("q_out", q_out)) + ((("pold", pold),) if pold is not None else ()):
            if not (a.is_cuda and a.dtype == torch.float32 and a.is_contiguous() and a.numel() == self.N):
                raise ValueError(f"apply_inner: {name} must be a contiguous float32 CUDA tensor of {self.N} elements")
        pq = C.c_double(0.0)
        _check(load().rf_apply_inner(self.ctx, C.c_void_p(z.data_ptr()),
                                     None if pold is None else C.c_void_p(pold.data_ptr()), float(beta),
                                     C.c_void_p(p_out.data_ptr()), C.c_void_p(q_out.data_ptr()), C.byref(pq)),
               "rf_apply_inner")
        return pq.value

    def set_wait_limit(self, polls: int):
        """Test hook of the bounded device waits (0: default; < 0: one non-blocking test)."""
        _check(load().rf_set_wait_limit(self.ctx, int(polls)), "rf_set_wait_limit")

    # -- learned warm start
    def ws_features(self, scales: "rf_ws_scales", t: float, dt: float, out, h=None):
        """Network features of state h (device, N doubles; None = current state) for a step dt
        from time t into out (N x 4 float32, device)."""
        _check(load().rf_ws_features(self.ctx, C.byref(scales), None if h is None else C.c_void_p(h.data_ptr()),
                                     float(t), float(dt), C.c_void_p(out.data_ptr())), "rf_ws_features")

    def ws_target(self, scales: "rf_ws_scales", h_old, dt: float, target, mask=None):
        _check(load().rf_ws_target(self.ctx, C.byref(scales), C.c_void_p(h_old.data_ptr()), float(dt),
                                   C.c_void_p(target.data_ptr()),
                                   None if mask is None else C.c_void_p(mask.data_ptr())), "rf_ws_target")

    def ws_attach(self, net: Optional["Network"], scales: Optional["rf_ws_scales"] = None):
        self._ws_net = net   # keep the network alive while attached
        _check(load().rf_ws_attach(self.ctx, None if net is None else net.handle,
                                   None if scales is None else C.byref(scales)), "rf_ws_attach")

    def ws_stats(self) -> dict:
        st = rf_ws_stats()
        _check(load().rf_ws_get_stats(self.ctx, C.byref(st)), "rf_ws_get_stats")
        return {"guesses": st.guesses, "fallbacks": st.fallbacks}


class Network:
    """The warm-start network (BF16 3-D conv residual net) on the current device and torch stream."""

    def __init__(self, stream=None, use_torch_allocator=True):
        import torch
        L = load()
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._allocator = TorchAllocator(self.device) if use_torch_allocator else None
        h = _VP()
        _check(L.rf_nn_create(C.c_void_p(self.stream.cuda_stream),
                              C.byref(self._allocator.struct) if self._allocator else None, C.byref(h)),
               "rf_nn_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            load().rf_nn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        a = np.ascontiguousarray(theta, dtype=np.float32)
        _check(load().rf_nn_set_params(self.handle, a.ctypes.data_as(_VP), a.size), "rf_nn_set_params")

    def get_params(self) -> np.ndarray:
        a = np.empty(NN_PARAMS, dtype=np.float32)
        _check(load().rf_nn_get_params(self.handle, a.ctypes.data_as(_VP), a.size), "rf_nn_get_params")
        return a

    @staticmethod
    def _dims(x):
        B, D, H, W, c = x.shape
        assert c == 4 and x.is_contiguous()
        return B, D, H, W

    def forward(self, x, y):
        """x: (B, D, H, W, 4) float32 device tensor; y: (B, D, H, W) float32."""
        B, D, H, W = self._dims(x)
        _check(load().rf_nn_forward(self.handle, C.c_void_p(x.data_ptr()), B, D, H, W, C.c_void_p(y.data_ptr())),
               "rf_nn_forward")

    def loss_grad(self, x, target, mask=None, want_grad=True):
        B, D, H, W = self._dims(x)
        loss = C.c_float(0.0)
        g = np.empty(NN_PARAMS, dtype=np.float32) if want_grad else None
        _check(load().rf_nn_loss_grad(self.handle, C.c_void_p(x.data_ptr()), C.c_void_p(target.data_ptr()),
                                      None if mask is None else C.c_void_p(mask.data_ptr()), B, D, H, W,
                                      C.byref(loss), None if g is None else g.ctypes.data_as(_VP)),
               "rf_nn_loss_grad")
        return loss.value, g

    def train_step(self, x, target, mask=None, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, want_loss=True):
        B, D, H, W = self._dims(x)
        opt = rf_adam(lr, beta1, beta2, eps)
        loss = C.c_float(0.0)
        _check(load().rf_nn_train_step(self.handle, C.c_void_p(x.data_ptr()), C.c_void_p(target.data_ptr()),
                                       None if mask is None else C.c_void_p(mask.data_ptr()), B, D, H, W,
                                       C.byref(opt), C.byref(loss) if want_loss else None), "rf_nn_train_step")
        return loss.value if want_loss else None

    def launch_count(self) -> int:
        return int(load().rf_nn_launch_count(self.handle))

    def set_trace(self, on: bool = True):
        _check(load().rf_nn_set_trace(self.handle, 1 if on else 0), "rf_nn_set_trace")

    TRACE = {"input": (0, 8, "bf16"), "block_out": (1, 32, "bf16"), "block_mid": (2, 32, "bf16"),
             "out_grad": (3, 32, "bf16"), "output": (4, 8, "f32")}

    def trace_get(self, what: str, index: int, shape):
        """A stored tensor of the last traced gradient evaluation as float64,
        shape (B, D, H, W, channels)."""
        code, ch, kind = self.TRACE[what]
        if what == "out_grad" and index == NN_LAYERS - 1:
            ch = 8
        M = int(np.prod(shape))
        buf = np.empty(M * ch, dtype=np.uint16 if kind == "bf16" else np.float32)
        _check(load().rf_nn_trace_get(self.handle, code, int(index), buf.ctypes.data_as(_VP), buf.size),
               "rf_nn_trace_get")
        if kind == "bf16":
            buf = (buf.astype(np.uint32) << 16).view(np.float32)
        return buf.astype(np.float64).reshape(tuple(shape) + (ch,))


class Ensemble:
    """A batched ensemble of independent instances (rf_ens_*)."""

    def __init__(self, instances, params=None, stream=None, use_torch_allocator=True):
        import torch
        L = load()
        self.n = len(instances)
        arr = (rf_ens_instance * self.n)(*instances)
        self.params = params if params is not None else default_params()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._allocator = TorchAllocator(torch.device("cuda", torch.cuda.current_device())) \
            if use_torch_allocator else None
        h = _VP()
        _check(L.rf_ens_create(arr, self.n, C.byref(self.params), C.c_void_p(self.stream.cuda_stream),
                               C.byref(self._allocator.struct) if self._allocator else None, C.byref(h)),
               "rf_ens_create")
        self.ctx = h
        self.cells = [i.nx * i.ny * i.nz for i in instances]

    @staticmethod
    def instance_of_case(case) -> rf_ens_instance:
        """A workloads.Case with one soil, uniform initial head, top/bottom
        conditions and zero-flux lateral faces as an ensemble instance."""
        s = case.soils[0]
        soil = rf_soil(MODELS[s.get("model", "vg")], s["theta_r"], s["theta_s"], s["alpha"], s.get("n", 2.0),
                       s["Ks"], s.get("S", 1e-5))
        top = next((b for b in case.bcs if b.face == "zmax"), None)
        bot = next((b for b in case.bcs if b.face == "zmin"), None)
        tt, tv = (BC_TYPES[top.type], float(top.v[0]) if top.v is not None else 0.0) if top else (0, 0.0)
        bt, bv = (BC_TYPES[bot.type], float(bot.v[0]) if bot.v is not None else 0.0) if bot else (0, 0.0)
        return rf_ens_instance(case.nx, case.ny, case.nz, case.dx, case.dy, case.dz, soil, float(case.h0[0]),
                               tt, tv, bt, bv)

    @classmethod
    def from_cases(cls, cases, **param_overrides):
        p = dict(cases[0].params)
        p.update(param_overrides)
        return cls([cls.instance_of_case(c) for c in cases], params=default_params(**p))

    def close(self):
        if getattr(self, "ctx", None):
            load().rf_ens_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tiling(self, cluster: int, threads: int = 512):
        _check(load().rf_ens_set_tiling(self.ctx, int(cluster), int(threads)), "rf_ens_set_tiling")

    def set_schedule(self, order=None, n_wide: int = -1):
        """Queue order (instance indices; None = largest first) and how many
        leading instances run on whole clusters (-1 = all)."""
        arr = None
        if order is not None:
            order = [int(i) for i in order]
            arr = (C.c_int * len(order))(*order)
        _check(load().rf_ens_set_schedule(self.ctx, arr, int(n_wide)), "rf_ens_set_schedule")

    def run(self, t_end):
        _check(load().rf_ens_run(self.ctx, float(t_end)), "rf_ens_run")

    def get(self, i, want_h=True):
        st = rf_ens_stats()
        h = np.zeros(self.cells[i]) if want_h else None
        _check(load().rf_ens_get(self.ctx, int(i), _dptr(h), C.byref(st)), "rf_ens_get")
        return h, {k: getattr(st, k) for k, _ in rf_ens_stats._fields_}

    def reset(self):
        _check(load().rf_ens_reset(self.ctx), "rf_ens_reset")

    def tune(self, t_probe):
        """Tile and schedule; returns (cluster, threads, n_wide, ms) of the fastest."""
        c, th, w, ms = C.c_int(0), C.c_int(0), C.c_int(0), C.c_double(0)
        _check(load().rf_ens_tune(self.ctx, float(t_probe), C.byref(c), C.byref(th), C.byref(w), C.byref(ms)),
               "rf_ens_tune")
        return c.value, th.value, w.value, ms.value


def ens_model_makespan(wide_s, order, units, cluster=1, n_wide=None, solo_s=None) -> float:
    """The ensemble tuner's list-scheduling model (host arithmetic, no GPU)."""
    w = np.ascontiguousarray(wide_s, dtype=np.float64)
    so = None if solo_s is None else np.ascontiguousarray(solo_s, dtype=np.float64)
    o = np.ascontiguousarray(order, dtype=np.int32)
    n = len(w)
    out = C.c_double(0.0)
    _check(load().rf_ens_model_makespan(_dptr(w), _dptr(so), o.ctypes.data_as(C.POINTER(C.c_int)), n,
                                        n if n_wide is None else int(n_wide), int(units), int(cluster),
                                        C.byref(out)), "rf_ens_model_makespan")
    return out.value


def pcg_solve_noalloc(shape, diag, Tx, Ty, Tz, b, x, tol=1e-10, max_it=10000, stream=None) -> int:
    """rf_pcg_solve_noalloc on torch CUDA float64 tensors (x in/out)."""
    import torch
    nx, ny, nz = shape
    n = int(nx) * int(ny) * int(nz)
    dev = torch.cuda.current_device()
    for name, a in (("diag", diag), ("Tx", Tx), ("Ty", Ty), ("Tz", Tz), ("b", b), ("x", x)):
        # a short, strided or float32 tensor would be read out of bounds on the device
        if not (isinstance(a, torch.Tensor) and a.is_cuda and a.device.index == dev and a.dtype == torch.float64
                and a.is_contiguous() and a.numel() == n):
            raise ValueError(f"pcg_solve_noalloc: {name} must be a contiguous float64 CUDA tensor of "
                             f"{n} elements on the current device")
    st = stream if stream is not None else torch.cuda.current_stream()
    it = C.c_int(0)
    ptr = lambda a: C.c_void_p(a.data_ptr())
    _check(load().rf_pcg_solve_noalloc(nx, ny, nz, ptr(diag), ptr(Tx), ptr(Ty), ptr(Tz), ptr(b), ptr(x), float(tol),
                                       int(max_it), C.c_void_p(st.cuda_stream), C.byref(it)), "rf_pcg_solve_noalloc")
    return it.value


def header_function_names(header: str) -> list:
    """Names of the functions declared in include/rf.h."""
    import re
    txt = open(header).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rf_[a-z_0-9]+)\s*\(", txt)))
