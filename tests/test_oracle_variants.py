"""Pins of the oracle's variants beyond the paper's default scheme.

Gravity direction (Eq. 1's elevation gradient in the grid's axes, for a grid
aligned with a tilted slab, as in the paper's slope of Sec. 4.2): the same
column laid along x, y or z with gravity along its axis gives the same
solution step for step; a hydrostatic head h = c - z_e(x) under a tilted
gravity is a fixed point with zero-flux faces; the tilted-slope workload
closes its balance and is uniform along a level river.

Interface conductivity: the harmonic mean reproduces the closed-form steady
state across layers (series resistance), the arithmetic mean of Sec. 2.2
does not.

Brooks-Corey closure (the alternative Sec. 1 names): closed forms, C as
d(theta)/dh, continuity at the air-entry head, a mass-conserving run.

Richardson step-doubling time control (the alternative to EBATS Sec. 2.2
names): the error estimate is second order in dt, accepted steps respect the
tolerance, the global error falls with it.

Variable-step BDF2 (the multistep alternative Sec. 2.2 names): second order
in time where backward Euler is first order."""
import numpy as np
import pytest

from oracle import oracle as O

SOIL = dict(model=O.VG, theta_r=0.078, theta_s=0.43, alpha=3.6, n=1.56, Ks=2.89e-6, S=1e-5)
FACES = {"x": (O.XMIN, O.XMAX), "y": (O.YMIN, O.YMAX), "z": (O.ZMIN, O.ZMAX)}


def _column(axis, n=40, d=0.01):
    shape = {"x": (n, 1, 1), "y": (1, n, 1), "z": (1, 1, n)}[axis]
    size = {"x": (d, 1.0, 1.0), "y": (1.0, d, 1.0), "z": (1.0, 1.0, d)}[axis]
    o = O.Oracle(*shape, *size, 0.0, None)
    o.set_soils([SOIL], None, None)
    lo, hi = FACES[axis]
    o.set_bc(lo, O.DIRICHLET, np.array([0.0]), np.array([-1.0]))
    o.set_bc(hi, O.DIRICHLET, np.array([0.0]), np.array([-0.05]))
    grav = {"x": (1.0, 0.0, 0.0), "y": (0.0, 1.0, 0.0), "z": (0.0, 0.0, 1.0)}[axis]
    o.set_params(grav_x=grav[0], grav_y=grav[1], grav_z=grav[2], tol_cg=1e-13)
    o.set_state(np.full(n, -1.0), 0.0)
    return o


def test_column_along_any_axis_is_the_same_column():
    runs = {}
    for axis in "xyz":
        o = _column(axis)
        steps = o.run(1800.0)
        runs[axis] = (o.get_state()[0], [(s.dt, s.picard, s.rejected) for s in steps], o.mass_balance())
    for axis in "xy":
        assert runs[axis][1] == runs["z"][1]
        np.testing.assert_allclose(runs[axis][0], runs["z"][0], rtol=0, atol=1e-11)
        assert runs[axis][2]["inflow_cum"] == pytest.approx(runs["z"][2]["inflow_cum"], rel=1e-10)
    # the infiltration moved water: the test is not trivially static
    assert np.max(np.abs(runs["z"][0] + 1.0)) > 0.1


def test_tilted_hydrostatic_head_is_a_fixed_point():
    a, b = np.radians(20.0), np.radians(3.0)
    g = np.array([np.sin(a), np.cos(a) * np.sin(b), np.cos(a) * np.cos(b)])   # unit elevation gradient
    nx, ny, nz, d = 6, 5, 4, (2.0, 2.0, 0.2)
    o = O.Oracle(nx, ny, nz, *d, 0.0, None)
    o.set_soils([SOIL], None, None)                # every face zero flux (the default)
    o.set_params(grav_x=g[0], grav_y=g[1], grav_z=g[2])
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ze = g[0] * (i + 0.5) * d[0] + g[1] * (j + 0.5) * d[1] + g[2] * (k + 0.5) * d[2]
    h0 = (-0.5 - ze).ravel()
    o.set_state(h0, 0.0)
    steps = o.run(86400.0)
    assert np.max(np.abs(o.get_state()[0] - h0)) <= 1e-9
    assert all(s.picard == 1 for s in steps)
    mb = o.mass_balance()
    assert mb["inflow_cum"] == 0.0 and mb["outflow_cum"] == 0.0


def test_tilted_slope_workload_in_the_oracle():
    # a small piece of the Sec. 4.2 slope for one day: the balance closes;
    # a level river (no slope along y) leaves the solution uniform along y,
    # the 3 degree river does not
    from paper_1809_10895_gb300 import workloads as W
    from tests.helpers import oracle_from_case
    spread = {}
    for rd in (0.0, 3.0):
        c = W.tilted_slope(nx=24, ny=6, nz=10, river_deg=rd, days=1.0)
        o = oracle_from_case(c)
        o.run(c.t_end)
        h = o.get_state()[0].reshape(c.nz, c.ny, c.nx)
        spread[rd] = np.max(np.ptp(h, axis=1))
        mb = o.mass_balance()
        assert mb["closure_rel"] <= 1e-9
        assert mb["inflow_cum"] > 0.0
    assert spread[0.0] <= 1e-9
    assert spread[3.0] >= 1e-5


def test_harmonic_face_mean_gives_the_exact_layered_steady_state():
    # saturated steady flow across two layers (Ks 1e-5 over 1e-7 m/s), heads
    # held at both ends: the exact solution is linear in total head within
    # each layer with the series resistance 0.5/K1 + 0.5/K2 (closed form);
    # the harmonic interface mean reproduces it at the cell centres, the
    # arithmetic mean of Sec. 2.2 does not at the interface
    nz, dz, K1, K2 = 20, 0.05, 1e-5, 1e-7
    zc = (np.arange(nz) + 0.5) * dz
    Hb, Ht = 2.0 + 0.0, 0.5 + nz * dz
    q = (Hb - Ht) / (0.5 / K1 + 0.5 / K2)
    H = np.where(zc <= 0.5, Hb - q * zc / K1, Hb - q * 0.5 / K1 - q * (zc - 0.5) / K2)
    exact = H - zc
    err = {}
    for fm in (0, 1):
        o = O.Oracle(1, 1, nz, 1.0, 1.0, dz, 0.0, None)
        soil = dict(model=O.VG, theta_r=0.05, theta_s=0.4, alpha=2.0, n=1.8, Ks=K1, S=1e-4)
        o.set_soils([soil, dict(soil, Ks=K2)], np.array([0] * 10 + [1] * 10, np.uint8), None)
        o.set_bc(O.ZMIN, O.DIRICHLET, np.array([0.0]), np.array([2.0]))
        o.set_bc(O.ZMAX, O.DIRICHLET, np.array([0.0]), np.array([0.5]))
        o.set_params(face_mean=fm, dt_max=1e6, tol_cg=1e-14)
        o.set_state(np.full(nz, 2.0), 0.0)
        o.run(3e8)
        err[fm] = np.max(np.abs(o.get_state()[0] - exact))
    assert err[1] <= 1e-9
    assert err[0] >= 1e-4


BC_SOIL = dict(model=O.BROOKS_COREY, theta_r=0.05, theta_s=0.40, alpha=1 / 0.3, n=0.5, Ks=1e-5, S=1e-5)


def test_brooks_corey_closed_forms():
    # Brooks and Corey (the alternative closure named in Sec. 1): at twice the
    # air-entry head Se = 2^-lambda, K = Ks 2^-(2 + 3 lambda); theta_s and Ks
    # above the air-entry head; theta_r and 0 far below it
    hb, lam = -0.3, 0.5
    th, K, C = O.closure(BC_SOIL, 2 * hb)
    assert th == pytest.approx(0.05 + 0.35 * 2 ** -lam, rel=1e-14)
    assert K == pytest.approx(1e-5 * 2 ** -(2 + 3 * lam), rel=1e-13)
    th, K, C = O.closure(BC_SOIL, 0.5 * hb)
    assert (th, K, C) == (0.40, 1e-5, 0.0)
    th, K, _ = O.closure(BC_SOIL, hb * (1 + 1e-12))
    assert th == pytest.approx(0.40, rel=1e-10) and K == pytest.approx(1e-5, rel=1e-10)
    th, K, _ = O.closure(BC_SOIL, -1e8)
    assert th == pytest.approx(0.05, abs=1e-4) and K < 1e-20


@pytest.mark.parametrize("h", [-0.31, -0.5, -2.0, -30.0])
def test_brooks_corey_capacity_is_dtheta_dh(h):
    e = 1e-6 * abs(h)
    fd = (O.closure(BC_SOIL, h + e)[0] - O.closure(BC_SOIL, h - e)[0]) / (2 * e)
    assert O.closure(BC_SOIL, h)[2] == pytest.approx(fd, rel=1e-6)


def test_brooks_corey_column_conserves_mass():
    # wetting from a top head below the air-entry head (lambda 2): no
    # rejection, the balance closes, water enters
    o = O.Oracle(1, 1, 50, 1.0, 1.0, 0.02, 0.0, None)
    o.set_soils([dict(BC_SOIL, n=2.0)], None, None)
    o.set_bc(O.ZMAX, O.DIRICHLET, np.array([0.0]), np.array([-0.5]))
    o.set_bc(O.ZMIN, O.FREE_DRAINAGE)
    o.set_params(tol_cg=1e-12)
    o.set_state(np.full(50, -2.0), 0.0)
    steps = o.run(3600.0)
    mb = o.mass_balance()
    assert sum(s.rejected for s in steps) == 0
    assert mb["closure_rel"] <= 1e-11
    assert mb["inflow_cum"] > 0.0


def _column_state():
    from paper_1809_10895_gb300 import workloads as W
    from tests.helpers import oracle_from_case
    case = W.infiltration_column(nz=60, dz=0.01, t_end=3600.0)
    o = oracle_from_case(case)
    o.run(600.0)
    return case, oracle_from_case, o.get_state()


def test_richardson_estimate_is_second_order():
    # the step-doubling estimate of backward Euler's local error scales as dt^2
    case, mk, (h0, meta) = _column_state()
    errs = []
    for dt in (8.0, 4.0, 2.0):
        q = mk(case, time_control=1, tol_time=1e9, dt0=dt)
        q.set_state(h0, meta["t"])
        assert q.step().dt == dt
        errs.append(q.time_error(largest=False))
    for a, b in zip(errs, errs[1:]):
        assert 3.0 <= a / b <= 5.0


def test_richardson_control_bounds_the_error():
    # every accepted step's estimate is within tol; the error against a fine
    # fixed-dt reference shrinks with tol; the balance closes
    case, mk, (h0, meta) = _column_state()
    ref = mk(case, dt0=0.25, f_grow=1.0)
    ref.set_state(h0, meta["t"])
    ref.run(meta["t"] + 600.0)
    hr = ref.get_state()[0]
    glob = {}
    for tol in (1e-2, 1e-4):
        q = mk(case, time_control=1, tol_time=tol, dt0=1.0)
        q.set_state(h0, meta["t"])
        q.run(meta["t"] + 600.0)
        assert q.time_error() <= tol
        assert q.mass_balance()["closure_rel"] <= 1e-9
        glob[tol] = np.max(np.abs(q.get_state()[0] - hr))
    assert glob[1e-4] < 0.5 * glob[1e-2]


LOAM_O = dict(model=O.VG, theta_r=0.078, theta_s=0.43, alpha=3.6, n=1.56, Ks=2.89e-6, S=1e-5)


def _fixed_dt_column(scheme, dt, T=1800.0, picard_form=1):
    o = O.Oracle(1, 1, 40, 1.0, 1.0, 0.025, 0.0, None)
    o.set_soils([LOAM_O], None, None)
    o.set_bc(O.ZMAX, O.DIRICHLET, np.array([0.0]), np.array([-0.3]))
    o.set_bc(O.ZMIN, O.FREE_DRAINAGE)
    o.set_params(picard_form=picard_form, time_scheme=scheme, dt0=dt, dt_max=dt, f_grow=1.0, tol_picard=1e-11,
                 tol_cg=1e-14)
    o.set_state(np.full(40, -1.0), 0.0)
    steps = o.run(T)
    assert all(s.rejected == 0 for s in steps)
    return o.get_state()[0], o.mass_balance()


def test_bdf2_is_second_order_and_backward_euler_first():
    # variable-step BDF2 (the multistep alternative Sec. 2.2 names), mixed
    # form: halving dt divides the error at t = 30 min by ~4; backward Euler
    # by ~2 (reference: BDF2 at dt = 0.94 s)
    ref, _ = _fixed_dt_column(1, 0.9375)
    err = {}
    for scheme in (0, 1):
        err[scheme] = []
        for dt in (30.0, 15.0, 7.5):
            h, mb = _fixed_dt_column(scheme, dt)
            assert mb["closure_rel"] <= 1e-9
            err[scheme].append(np.max(np.abs(h - ref)))
    for a, b in zip(err[0], err[0][1:]):
        assert 1.7 <= a / b <= 2.3
    for a, b in zip(err[1], err[1][1:]):
        assert 3.4 <= a / b <= 4.6
    assert err[1][1] < 0.1 * err[0][1]


def test_bdf2_needs_the_mixed_form():
    with pytest.raises(RuntimeError):
        _fixed_dt_column(1, 30.0, picard_form=0)
