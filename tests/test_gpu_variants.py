"""GPU-vs-oracle parity of the scheme's variants, through the C ABI.

Each variant runs on the CUDA path and in the CPU oracle on the same seeded
inputs; the step sequences (dt, Picard counts, reruns) are identical and the
heads agree within 1e-8 m on the FP64 path (1e-6 m on the mixed path), with
the water balance closed:

* gravity along tilted grid axes (the slope of Sec. 4.2 on a slab-aligned
  grid), FP64 and mixed paths;
* the Brooks-Corey closure (the alternative Sec. 1 names);
* the harmonic interface conductivity (Sec. 2.2's interpolation
  alternative);
* variable-step BDF2 in the mixed form (the multistep alternative of
  Sec. 2.2);
* Richardson step-doubling time control (Sec. 2.2's alternative to EBATS);
* double-float closures on the FP64 path and FP64 closures on the mixed path.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1809_10895_gb300 import rf
from paper_1809_10895_gb300 import workloads as W
from tests.helpers import oracle_from_case

pytestmark = pytest.mark.gpu

TOL_PLAIN = 1e-8
TOL_MIXED = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1809_10895_gb300 import build as B
    B.build()
    rf.load()
    torch.cuda.set_device(0)


GPU_ONLY = ("precision", "tol_inner", "closure_arith", "precond")


def _run_pair(case, t_end, **over):
    s = rf.Solver.from_case(case, **over)
    o = oracle_from_case(case, **{k: v for k, v in over.items() if k not in GPU_ONLY})
    sg = s.run(t_end)
    so = o.run(t_end)
    return s, o, sg, so


def _check(case, s, o, sg, so, tol, closure=1e-9, dt_rtol=0.0):
    assert len(sg) == len(so) and len(sg) > 3
    if dt_rtol == 0.0:
        assert np.array_equal([a.dt for a in sg], [b.dt for b in so])
    else:
        np.testing.assert_allclose([a.dt for a in sg], [b.dt for b in so], rtol=dt_rtol, atol=0)
    assert [a.picard for a in sg] == [b.picard for b in so]
    assert [a.rejected for a in sg] == [b.rejected for b in so]
    hg, _ = s.get_state()
    ho, _ = o.get_state()
    act = np.ones(case.N, bool) if case.active is None else case.active.astype(bool)
    assert np.max(np.abs(hg - ho)[act]) <= tol
    mbg, mbo = s.mass_balance(), o.mass_balance()
    assert mbg["closure_rel"] <= closure
    for k in ("storage", "inflow_cum", "outflow_cum"):
        assert abs(mbg[k] - mbo[k]) <= 1e-9 * (mbo["storage0"] + abs(mbo[k]))


def _small_box(seed=7, **kw):
    return W.heterogeneous_box(20, 13, 12, d=0.25, seed=seed, water_table_depth=1.5, rain=5e-6, rain_hours=1.0,
                               t_end=3 * 3600.0, tol_cg=1e-13, **kw)


@pytest.mark.parametrize("precision,tol", [("fp64", TOL_PLAIN), ("mixed", TOL_MIXED)])
def test_tilted_slope_gravity(precision, tol):
    # the slope of Sec. 4.2 (20 degrees, river at 3 degrees) on a small
    # slab-aligned grid: river face Dirichlet 0, rain on the top face
    case = W.tilted_slope(nx=20, ny=8, nz=10, days=0.25, tol_cg=1e-13)
    s, o, sg, so = _run_pair(case, case.t_end, precision=precision)
    _check(case, s, o, sg, so, tol)
    assert s.mass_balance()["inflow_cum"] > 0.0


def test_tilted_hydrostatic_head_is_a_fixed_point_on_the_gpu():
    # h = c - z_e with z_e the elevation along the tilted axes, zero-flux faces
    g = (np.sin(0.3), np.cos(0.3) * np.sin(0.1), np.cos(0.3) * np.cos(0.1))
    case = W.Case(name="tilted_hydro", nx=12, ny=6, nz=8, dx=0.5, dy=0.5, dz=0.1, gravity=g,
                  soils=[dict(W.LOAM)], params=W.default_params(tol_cg=1e-13))
    i = np.tile(np.arange(12), 6 * 8)
    j = np.tile(np.repeat(np.arange(6), 12), 8)
    k = np.repeat(np.arange(8), 72)
    ze = g[0] * (i + 0.5) * 0.5 + g[1] * (j + 0.5) * 0.5 + g[2] * (k + 0.5) * 0.1
    case.h0 = 2.0 - ze
    s = rf.Solver.from_case(case)
    steps = s.run(3600.0)
    assert all(x.picard == 1 for x in steps)
    assert np.max(np.abs(s.get_state()[0] - case.h0)) <= 1e-12


def test_brooks_corey_closure():
    case = W.Case(name="bc_box", nx=10, ny=7, nz=14, dx=0.2, dy=0.2, dz=0.05,
                  soils=[dict(model="brooks_corey", theta_r=0.05, theta_s=0.40, alpha=2.0, n=0.8, Ks=1e-5, S=1e-5)],
                  Ks_cell=np.exp(np.log(1e-5) + 0.5 * np.random.default_rng(3).standard_normal(980)),
                  params=W.default_params(tol_cg=1e-13))
    case.h0 = np.linspace(-2.5, -1.0, case.N)
    case.bcs = [W.BC("zmax", "flux", np.array([0.0, 3600.0]), np.array([4e-6, 0.0])),
                W.BC("zmin", "dirichlet", np.array([0.0]), np.array([-2.0]))]
    s, o, sg, so = _run_pair(case, 2 * 3600.0)
    _check(case, s, o, sg, so, TOL_PLAIN)


def test_harmonic_interface_mean():
    case = _small_box(seed=9, face_mean=1)
    s, o, sg, so = _run_pair(case, case.t_end)
    _check(case, s, o, sg, so, TOL_PLAIN)
    # the interface mean matters on this field: the arithmetic run differs
    a = rf.Solver.from_case(case, face_mean=0)
    a.run(case.t_end)
    assert np.max(np.abs(a.get_state()[0] - s.get_state()[0])) > 1e-4


@pytest.mark.parametrize("precision,tol", [("fp64", TOL_PLAIN), ("mixed", TOL_MIXED)])
def test_bdf2_time_scheme(precision, tol):
    case = _small_box(seed=11, picard_form=1, time_scheme=1)
    s, o, sg, so = _run_pair(case, case.t_end, precision=precision)
    _check(case, s, o, sg, so, tol)


def test_richardson_time_control():
    # the next dt is a continuous function of the error estimate, a difference
    # of two solutions each known to the CG tolerance: GPU and oracle agree on
    # it to about 1e-7 relative, not bit for bit as under EBATS's discrete
    # factors; Picard counts and reruns stay identical
    case = _small_box(seed=13, time_control=1, tol_time=2e-3)
    s, o, sg, so = _run_pair(case, case.t_end)
    _check(case, s, o, sg, so, TOL_PLAIN, dt_rtol=1e-5)
    # the controller moved dt (neither EBATS' sequence nor a constant)
    dts = [x.dt for x in sg]
    assert len(set(np.round(dts, 9))) > 3


@pytest.mark.parametrize("precision,arith,tol", [("fp64", "double_float", TOL_PLAIN), ("mixed", "fp64", TOL_MIXED)])
def test_closure_arithmetic_options(precision, arith, tol):
    case = _small_box(seed=15)
    s, o, sg, so = _run_pair(case, case.t_end, precision=precision, closure_arith=arith)
    _check(case, s, o, sg, so, tol)
