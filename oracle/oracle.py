"""ctypes wrapper around the plain FP64 CPU oracle (``richards_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package entry's
``smoke()`` check and by the benchmark's CPU-baseline leg, never by the
product library.  It shares no code with the CUDA path.

The oracle restates the method of Orgogozo et al. (arXiv:1809.10895):
Eq. 1-4, the Picard / chord-slope / backward-Euler / explicit-gravity scheme of
Sec. 2.2, the global Picard exit test of Sec. 2.3 and Appendix A's Gardner
model.  Everything here is argument marshalling.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "richards_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liboracle.so")
LIB_OMP = os.path.join(BUILD_DIR, "liboracle_omp.so")   # the same source built with -fopenmp

VG, GARDNER, BROOKS_COREY = 0, 1, 2
ZERO_FLUX, DIRICHLET, FLUX, FREE_DRAINAGE, SEEPAGE = range(5)
XMIN, XMAX, YMIN, YMAX, ZMIN, ZMAX = range(6)
SOLVER_PCG, SOLVER_DENSE, SOLVER_DIC, SOLVER_DIC_RB = 0, 1, 2, 3


def build(force: bool = False, openmp: bool = False):
    """Compile the oracle with gcc (portable C11, no FMA contraction).  With
    openmp, the same source with -fopenmp: its per-cell loops and sums run on
    all cores.  Returns the library path, or None when the OpenMP build is not
    possible here (the one-thread build is always required)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    out = LIB_OMP if openmp else LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(SRC):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared"] + (["-fopenmp"] if openmp else [])
        try:
            subprocess.check_call(cmd + ["-o", tmp, SRC, "-lm"],
                                  stderr=subprocess.DEVNULL if openmp else None)
        except (subprocess.CalledProcessError, OSError):
            if not openmp:
                raise
            return None
        os.replace(tmp, out)
    return out


_libs = {}


def _configure(L):
    dp, ip, u8p, vp = C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_uint8), C.c_void_p
    L.or_create.restype = vp
    L.or_create.argtypes = [C.c_int] * 3 + [C.c_double] * 4 + [u8p]
    L.or_destroy.argtypes = [vp]
    L.or_num_active.argtypes = [vp]
    L.or_num_threads.argtypes = []
    L.or_set_soils.argtypes = [vp, C.c_int, ip, dp, dp, dp, dp, dp, dp, u8p, dp]
    L.or_set_bc.argtypes = [vp, C.c_int, C.c_int, dp, dp, C.c_int]
    L.or_set_param.argtypes = [vp, C.c_char_p, C.c_double]
    L.or_set_state.argtypes = [vp, dp, C.c_double]
    L.or_get_state.argtypes = [vp, dp, dp]
    L.or_set_clock.argtypes = [vp, C.c_double, C.c_double, C.c_int]
    L.or_step.argtypes = [vp, dp]
    L.or_run.argtypes = [vp, C.c_double, dp, C.c_int, ip]
    L.or_mass_balance.argtypes = [vp, dp]
    L.or_assemble.argtypes = [vp, dp, dp, C.c_double, C.c_double, dp, dp, dp, dp, dp, ip, ip, dp, ip]
    L.or_solve.argtypes = [vp, dp, dp, C.c_double, C.c_double, dp, C.c_int, dp]
    L.or_spmv.argtypes = [vp, dp, dp, C.c_double, C.c_double, dp, dp]
    L.or_active_cells.argtypes = [vp, ip]
    L.or_closure_eval.argtypes = [C.c_int] + [C.c_double] * 7 + [dp]
    L.or_ebats_accept.argtypes = [dp, ip, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double]
    L.or_ebats_reject.argtypes = [dp, ip, C.c_double, C.c_double]
    L.or_time_error.argtypes = [vp, C.c_int]
    L.or_time_error.restype = C.c_double
    return L


def lib(openmp: bool = False):
    """The loaded oracle library (the OpenMP build with openmp; None when that
    build is not possible here)."""
    if openmp not in _libs:
        path = build(openmp=openmp)
        L = None
        if path is not None:
            try:
                L = _configure(C.CDLL(path))
            except OSError:                 # e.g. no OpenMP runtime to load
                if not openmp:
                    raise
        _libs[openmp] = L
    return _libs[openmp]


def num_threads(openmp: bool = False) -> int:
    """Threads the oracle's per-cell loops use (1 for the one-thread build)."""
    L = lib(openmp)
    return 0 if L is None else int(L.or_num_threads())


def _d(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_int))


def _u8(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_uint8))


def closure(soil: dict, h: float):
    """(theta*, K, C) at pressure head h for one soil (Eq. 2-4 / Eq. A6)."""
    out = np.zeros(3)
    lib().or_closure_eval(int(soil.get("model", VG)), soil["theta_r"], soil["theta_s"], soil["alpha"],
                          soil.get("n", 2.0), soil["Ks"], soil.get("S", 1e-5), float(h), _d(out))
    return out[0], out[1], out[2]


def gardner_steady_profile(z, q, Ks, alpha):
    """Appendix A, Eq. A8: steady pressure head of a Gardner column with the
    water table (h = 0) at z = 0 and a constant flux q at the top, q positive
    downward (infiltration), valid for -Ks e^{-alpha L}/(1 - e^{-alpha L}) < q < Ks:
    h(z) = ln[(q + (Ks - q) e^{-alpha z}) / Ks] / alpha."""
    import numpy as np
    z = np.asarray(z, dtype=np.float64)
    return np.log((q + (Ks - q) * np.exp(-alpha * z)) / Ks) / alpha


def ebats_accept(dt_nom, easy, picard, n_small, n_inc, f_grow, dt_max):
    d = C.c_double(dt_nom)
    e = C.c_int(easy)
    lib().or_ebats_accept(C.byref(d), C.byref(e), picard, n_small, n_inc, f_grow, dt_max)
    return d.value, e.value


def ebats_reject(dt_nom, easy, dt_attempted, f_shrink):
    d = C.c_double(dt_nom)
    e = C.c_int(easy)
    lib().or_ebats_reject(C.byref(d), C.byref(e), dt_attempted, f_shrink)
    return d.value, e.value


@dataclass
class StepInfo:
    dt: float
    t: float
    picard: int
    cg: int
    rejected: int
    max_dh: float


class OracleError(RuntimeError):
    pass


class Oracle:
    """A problem instance of the CPU oracle.  Arrays are numpy, cell order
    x fastest then y then z (index i + nx*(j + ny*k))."""

    def __init__(self, nx, ny, nz, dx, dy, dz, z_bottom=0.0, active=None, openmp=False):
        self._L = lib(openmp)
        if self._L is None:
            raise OracleError("the OpenMP build of the oracle is not available (gcc -fopenmp failed)")
        self.shape = (nx, ny, nz)
        self.N = nx * ny * nz
        act = None if active is None else np.ascontiguousarray(active, dtype=np.uint8).ravel()
        self._act = act
        self.h = self._L.or_create(nx, ny, nz, dx, dy, dz, z_bottom, _u8(act))
        if not self.h:
            raise OracleError("or_create failed")
        self.na = self._L.or_num_active(self.h)
        cells = np.zeros(self.na, dtype=np.int32)
        self._L.or_active_cells(self.h, _i(cells))
        self.active_cells = cells

    def __del__(self):
        if getattr(self, "h", None) and getattr(self, "_L", None) is not None:
            self._L.or_destroy(self.h)
            self.h = None

    @staticmethod
    def _check(st, what):
        if st != 0:
            raise OracleError(f"{what} failed with status {st}")

    def set_soils(self, soils, zone_of_cell=None, Ks_cell=None):
        nz = len(soils)
        model = np.array([s.get("model", VG) for s in soils], dtype=np.int32)
        cols = {k: np.array([s.get(k, dflt) for s in soils], dtype=np.float64)
                for k, dflt in (("theta_r", 0.0), ("theta_s", 0.4), ("alpha", 1.0), ("n", 2.0),
                                ("Ks", 1e-5), ("S", 1e-5))}
        z = None if zone_of_cell is None else np.ascontiguousarray(zone_of_cell, dtype=np.uint8).ravel()
        k = None if Ks_cell is None else np.ascontiguousarray(Ks_cell, dtype=np.float64).ravel()
        self._keep = (model, cols, z, k)
        self._check(self._L.or_set_soils(self.h, nz, _i(model), _d(cols["theta_r"]), _d(cols["theta_s"]),
                                       _d(cols["alpha"]), _d(cols["n"]), _d(cols["Ks"]), _d(cols["S"]),
                                       _u8(z), _d(k)), "set_soils")

    def set_bc(self, face, type_, t=None, v=None):
        if v is None:
            self._check(self._L.or_set_bc(self.h, face, type_, None, None, 0), "set_bc")
            return
        v = np.atleast_1d(np.asarray(v, dtype=np.float64))
        t = np.zeros(len(v)) if t is None else np.atleast_1d(np.asarray(t, dtype=np.float64))
        self._check(self._L.or_set_bc(self.h, face, type_, _d(t), _d(v), len(v)), "set_bc")

    def set_params(self, **kw):
        for k, v in kw.items():
            self._check(self._L.or_set_param(self.h, k.encode(), float(v)), f"set_param({k})")

    def set_state(self, h, t=0.0):
        h = np.ascontiguousarray(h, dtype=np.float64).ravel()
        self._check(self._L.or_set_state(self.h, _d(h), float(t)), "set_state")

    def set_clock(self, t, dt_nom, easy):
        """Time and EBATS counters of a saved state (after set_state)."""
        self._check(self._L.or_set_clock(self.h, float(t), float(dt_nom), int(easy)), "set_clock")

    def get_state(self):
        h = np.zeros(self.N)
        meta = np.zeros(4)
        self._L.or_get_state(self.h, _d(h), _d(meta))
        return h, dict(t=meta[0], dt_nom=meta[1], easy=int(meta[2]), n_active=int(meta[3]))

    def step(self) -> StepInfo:
        info = np.zeros(6)
        self._check(self._L.or_step(self.h, _d(info)), "step")
        return StepInfo(info[0], info[1], int(info[2]), int(info[3]), int(info[4]), info[5])

    def run(self, t_end, log_cap=1_000_000):
        log = np.zeros((max(log_cap, 1), 6))
        ns = C.c_int(0)
        st = self._L.or_run(self.h, float(t_end), _d(log), log_cap, C.byref(ns))
        steps = [StepInfo(r[0], r[1], int(r[2]), int(r[3]), int(r[4]), r[5]) for r in log[:min(ns.value, log_cap)]]
        self._check(st, "run")
        return steps

    def time_error(self, largest=True):
        """Richardson time control: the local error estimate of the largest
        accepted step since the state was set (largest=True), or of the last
        estimated step."""
        return self._L.or_time_error(self.h, 1 if largest else 0)

    def mass_balance(self):
        out = np.zeros(7)
        self._L.or_mass_balance(self.h, _d(out))
        keys = ("storage0", "storage", "inflow_cum", "outflow_cum", "closure_abs", "closure_rel",
                "nonlinear_defect_cum")
        return dict(zip(keys, out.tolist()))

    def assemble(self, hk, hn, dt, t=0.0, csr=False):
        """Per active cell K(h^k), theta*(h^k), c = V C^k/dt, b, diag; and the
        CSR matrix over active cells when csr=True."""
        na = self.na
        hk = np.ascontiguousarray(hk, dtype=np.float64).ravel()
        hn = np.ascontiguousarray(hn, dtype=np.float64).ravel()
        out = {k: np.zeros(na) for k in ("K", "theta", "c", "b", "diag")}
        rp = np.zeros(na + 1, dtype=np.int32) if csr else None
        col = np.zeros(7 * na, dtype=np.int32) if csr else None
        val = np.zeros(7 * na) if csr else None
        nnz = C.c_int(0)
        self._L.or_assemble(self.h, _d(hk), _d(hn), float(dt), float(t), _d(out["K"]), _d(out["theta"]),
                          _d(out["c"]), _d(out["b"]), _d(out["diag"]), _i(rp), _i(col), _d(val), C.byref(nnz))
        if csr:
            out["csr"] = (rp, col[:nnz.value].copy(), val[:nnz.value].copy())
        return out

    def solve(self, hk, hn, dt, t=0.0, x0=None, dense=False, method=None):
        """One linear solve of the system at (hk, hn, dt, t): Jacobi-PCG by
        default, dense Cholesky (dense=True) or method = SOLVER_* ."""
        hk = np.ascontiguousarray(hk, dtype=np.float64).ravel()
        hn = np.ascontiguousarray(hn, dtype=np.float64).ravel()
        x = (hk[self.active_cells] if x0 is None else np.asarray(x0, dtype=np.float64)).copy()
        res = C.c_double(0.0)
        m = SOLVER_DENSE if dense else (SOLVER_PCG if method is None else int(method))
        it = self._L.or_solve(self.h, _d(hk), _d(hn), float(dt), float(t), _d(x), m, C.byref(res))
        return x, it, res.value

    def spmv(self, hk, hn, dt, x, t=0.0):
        hk = np.ascontiguousarray(hk, dtype=np.float64).ravel()
        hn = np.ascontiguousarray(hn, dtype=np.float64).ravel()
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros(self.na)
        self._L.or_spmv(self.h, _d(hk), _d(hn), float(dt), float(t), _d(x), _d(y))
        return y
