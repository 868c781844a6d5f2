"""Pins of the oracle's discretisation, linear solver, Picard loop, EBATS and
mass balance against what the mathematics fixes independently of the code:

* hydrostatic head is an exact fixed point with zero flux (Appendix A, q = 0);
* saturated linear limit: K = Ks, C = S, so h - (z0 - z) obeys the heat
  equation; cosine modes are exact eigenvectors of the zero-flux cell-centred
  Laplacian, hence backward Euler scales them by 1/(1 + dt D lambda) per step;
* Appendix A: steady Gardner profile, Eq. A8 (sign of q read as downward
  positive), second-order convergence under refinement;
* unit-gradient steady state under free drainage with top flux K(h0);
* CG against the oracle's dense Cholesky and numpy's LU on tiny grids;
  symmetry and M-matrix structure;
* global water balance closes to the linear-solver tolerance;
* EBATS reproduces a hand-computed dt sequence (Sec. 2.2).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import oracle as O
from paper_1809_10895_gb300 import workloads as W
from tests.helpers import oracle_from_case

VG_SOIL = dict(model="vg", theta_r=0.05, theta_s=0.40, alpha=2.0, n=1.8, Ks=1e-5, S=1e-5)


def _box(nx, ny, nz, dx, dy, dz, soils, h0, bcs, params, **kw):
    c = W.Case(name="t", nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz, soils=soils, bcs=bcs,
               params=W.default_params(**params), h0=h0, **kw)
    return c


def test_hydrostatic_is_exact_fixed_point_3d():
    # mixed saturated/unsaturated heterogeneous block: water table mid-height,
    # bottom Dirichlet at the hydrostatic face value, all other faces no-flux
    nx, ny, nz, d = 5, 4, 12, 0.25
    rng = np.random.default_rng(3)
    Ks = np.exp(np.log(1e-5) + rng.standard_normal(nx * ny * nz))
    case = _box(nx, ny, nz, d, d, d, [VG_SOIL], None,
                [W.BC("zmin", "dirichlet", np.array([0.0]), np.array([1.5]))],
                dict(tol_cg=1e-13), Ks_cell=Ks)
    case.h0 = 1.5 - case.z_centres()          # water table at z = 1.5 m
    o = oracle_from_case(case)
    for _ in range(100):
        s = o.step()
        assert s.picard == 1
    h, meta = o.get_state()
    assert np.max(np.abs(h - case.h0)) <= 1e-12
    mb = o.mass_balance()
    assert abs(mb["storage"] - mb["storage0"]) <= 1e-12 * mb["storage0"]


@pytest.mark.parametrize("modes", [(0, 0, 1), (1, 2, 1), (2, 1, 3)])
def test_saturated_limit_decays_as_discrete_heat_equation(modes):
    # h = z0 - z + u with h > 0 everywhere: K = Ks and C = S exactly, gravity
    # cancels against the hydrostatic part, and u obeys S du/dt = Ks lap(u).
    # With zero-flux faces, prod cos(pi k (i+1/2)/N) is an exact eigenvector
    # of the cell-centred Laplacian with eigenvalue sum 4/d^2 sin^2(pi k/2N).
    nx, ny, nz = 6, 5, 8
    dx, dy, dz = 0.3, 0.2, 0.1            # unequal spacings catch a swapped A/d
    S, Ks = 1e-3, 2e-5
    soil = dict(VG_SOIL, S=S, Ks=Ks)
    kx, ky, kz = modes
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    u = (np.cos(np.pi * kx * (i + 0.5) / nx) * np.cos(np.pi * ky * (j + 0.5) / ny)
         * np.cos(np.pi * kz * (k + 0.5) / nz))
    u = np.ascontiguousarray(u.transpose(2, 1, 0)).ravel()
    dt = 20.0
    case = _box(nx, ny, nz, dx, dy, dz, [soil], None, [],
                dict(tol_cg=1e-14, tol_picard=1e-12, dt0=dt, dt_max=dt, f_grow=1.0))
    amp = 0.05
    base = (nz * dz + 1.0) - case.z_centres()
    case.h0 = base + amp * u
    o = oracle_from_case(case)
    lam = (4 / dx**2 * math.sin(math.pi * kx / (2 * nx)) ** 2
           + 4 / dy**2 * math.sin(math.pi * ky / (2 * ny)) ** 2
           + 4 / dz**2 * math.sin(math.pi * kz / (2 * nz)) ** 2)
    g = 1.0 / (1.0 + dt * (Ks / S) * lam)
    for n in range(1, 6):
        o.step()
        h, _ = o.get_state()
        expect = base + amp * g**n * u
        assert np.max(np.abs(h - expect)) <= 1e-10 * amp


def _gardner_steady(nz, q, t_end=6e5):
    L = 1.0
    soil = dict(model="gardner", theta_r=0.05, theta_s=0.40, alpha=0.06, Ks=1e-6, S=1e-5)
    case = _box(1, 1, nz, 1.0, 1.0, L / nz, [soil], None,
                [W.BC("zmin", "dirichlet", np.array([0.0]), np.array([0.0])),
                 W.BC("zmax", "flux", np.array([0.0]), np.array([q]))],
                dict(tol_cg=1e-13, tol_picard=1e-11, dt0=1.0, dt_max=2e4))
    zc = case.z_centres()
    case.h0 = -zc                                  # start hydrostatic
    case.t_end = t_end
    o = oracle_from_case(case)
    o.run(t_end)
    h, _ = o.get_state()
    Ks, a = 1e-6, 0.06
    exact = np.log((q + (Ks - q) * np.exp(-a * zc)) / Ks) / a      # Eq. A8
    return np.max(np.abs(h - exact))


@pytest.mark.parametrize("q", [-4e-6, -1e-6, 0.0, 5e-7, 9e-7])
def test_appendix_a_gardner_steady_state(q):
    # Eq. A8 with q the downward (infiltration-positive) flux; the flux must
    # satisfy -Ks e^-aL/(1-e^-aL) < q < Ks for an unsaturated column.
    e1 = _gardner_steady(25, q)
    e2 = _gardner_steady(50, q)
    if q == 0.0:
        assert e1 < 1e-9 and e2 < 1e-9            # hydrostatic: exact
    else:
        assert e2 < 2e-4
        assert e1 / e2 > 3.2                        # second order in dz


def test_unit_gradient_steady_state():
    # uniform h0, free-draining bottom and top flux K(h0): every face carries
    # the gravity flux K(h0) A_z, so nothing changes
    h0 = -0.6
    soil = VG_SOIL
    K0 = O.closure(dict(soil, model=O.VG), h0)[1]
    case = _box(3, 2, 30, 0.1, 0.1, 0.02, [soil], np.full(180, h0),
                [W.BC("zmax", "flux", np.array([0.0]), np.array([K0])), W.BC("zmin", "free_drainage")],
                dict(tol_cg=1e-14, dt_max=100.0))
    o = oracle_from_case(case)
    o.run(3600.0)
    h, _ = o.get_state()
    assert np.max(np.abs(h - h0)) <= 1e-12


def _tiny_system(seed=5):
    nx, ny, nz = 3, 4, 5
    rng = np.random.default_rng(seed)
    N = nx * ny * nz
    Ks = np.exp(np.log(1e-5) + rng.standard_normal(N))
    soils = [VG_SOIL, dict(VG_SOIL, alpha=3.0, n=1.4)]
    zone = (rng.random(N) < 0.5).astype(np.uint8)
    case = _box(nx, ny, nz, 0.2, 0.3, 0.1, soils, None,
                [W.BC("zmin", "dirichlet", np.array([0.0]), np.array([0.3])),
                 W.BC("zmax", "flux", np.array([0.0]), np.array([2e-6])),
                 W.BC("xmin", "dirichlet", np.array([0.0]), np.array([-0.5]))],
                dict(tol_cg=1e-14), Ks_cell=Ks, zone_of_cell=zone)
    case.h0 = -rng.uniform(0.05, 2.0, N)
    case.h0[:6] = rng.uniform(0.0, 0.2, 6)       # a few saturated cells
    hk = case.h0 + rng.normal(0, 0.05, N)
    return case, hk


def test_matrix_structure_and_dense_solvers():
    case, hk = _tiny_system()
    o = oracle_from_case(case)
    out = o.assemble(hk, case.h0, dt=30.0, csr=True)
    rp, col, val = out["csr"]
    A = sp.csr_matrix((val, col, rp), shape=(o.na, o.na)).toarray()
    assert np.allclose(A, A.T, rtol=0, atol=1e-18 * np.abs(A).max())
    off = A - np.diag(np.diag(A))
    assert np.all(off <= 0)
    # diagonally dominant, strictly by c = V C/dt (> 0)
    assert np.all(np.diag(A) - np.abs(off).sum(1) >= out["c"] * (1 - 1e-12))
    assert np.allclose(np.diag(A), out["diag"], rtol=1e-15)
    x_np = np.linalg.solve(A, out["b"])
    x_ch, it_ch, _ = o.solve(hk, case.h0, 30.0, dense=True)
    x_cg, it_cg, res = o.solve(hk, case.h0, 30.0)
    assert it_cg > 0
    scale = np.abs(x_np).max()
    assert np.max(np.abs(x_ch - x_np)) <= 1e-11 * scale
    assert np.max(np.abs(x_cg - x_np)) <= 1e-9 * scale
    # spmv is the same operator
    y = o.spmv(hk, case.h0, 30.0, x_np)
    assert np.allclose(y, A @ x_np, rtol=1e-13, atol=0)


def test_row_sums_equal_capacity_without_boundary_terms():
    # all faces zero-flux: A 1 = c (interior T cancel in each row)
    case, hk = _tiny_system()
    case.bcs = []
    o = oracle_from_case(case)
    out = o.assemble(hk, case.h0, dt=30.0, csr=True)
    rp, col, val = out["csr"]
    A = sp.csr_matrix((val, col, rp), shape=(o.na, o.na))
    assert np.allclose(A @ np.ones(o.na), out["c"], rtol=1e-9, atol=0)


def test_mass_balance_closes():
    case = W.heterogeneous_box(8, 7, 10, d=0.25, seed=1, t_end=4 * 3600.0, rain=5e-6, rain_hours=2.0,
                               water_table_depth=1.5, tol_cg=1e-13)
    o = oracle_from_case(case)
    steps = o.run(case.t_end)
    mb = o.mass_balance()
    assert len(steps) > 20
    assert mb["inflow_cum"] > 0 and mb["outflow_cum"] > 0
    assert mb["closure_rel"] <= 1e-11
    # bookkeeping identity: storage change = net inflow + nonlinear defect
    lhs = mb["storage"] - mb["storage0"]
    rhs = mb["inflow_cum"] - mb["outflow_cum"] + mb["nonlinear_defect_cum"]
    assert abs(lhs - rhs) <= 1e-12 * mb["storage0"]
    # the nonlinear defect is bounded by the Picard tolerance
    V = case.dx * case.dy * case.dz
    assert abs(mb["nonlinear_defect_cum"]) <= len(steps) * case.N * V * 0.5 * 1e-6


def test_ebats_scripted_sequence():
    # EBATS: grow by f after n_inc consecutive steps with <= n_small Picard
    # iterations (cap dt_max); a rejection divides the attempted dt by f and
    # resets the count.  Hand-computed sequence for f = 2, n_inc = 3.
    dt, easy = 1.0, 0
    seq = []
    for picard in [1, 2, 3, 1, 1, 4, 1, 1, 1, 2, 2, 2, 1, 1, 1]:
        dt, easy = O.ebats_accept(dt, easy, picard, 3, 3, 2.0, 5.0)
        seq.append((dt, easy))
    assert seq == [(1, 1), (1, 2), (2, 0), (2, 1), (2, 2), (2, 0), (2, 1), (2, 2), (4, 0),
                   (4, 1), (4, 2), (5, 0), (5, 1), (5, 2), (5, 0)]
    dt, easy = O.ebats_reject(5.0, 2, 3.0, 2.0)      # attempted (clipped) 3 s
    assert (dt, easy) == (1.5, 0)


def test_step_clipping_to_forcing_breakpoints():
    # each step sees one value of the piecewise-constant rain series: the
    # step ending at the breakpoint 7 s is clipped and the nominal dt is kept
    case = W.heterogeneous_box(4, 4, 6, d=0.25, seed=2, rain=1e-6, rain_hours=7.0 / 3600.0,
                               water_table_depth=1.0, dt0=3.0, dt_max=3.0)
    o = oracle_from_case(case)
    steps = o.run(13.0)
    assert [round(s.t, 12) for s in steps] == [3.0, 6.0, 7.0, 10.0, 13.0]
    _, meta = o.get_state()
    assert meta["dt_nom"] == 3.0


def test_infiltration_column_runs_and_conserves_mass():
    case = W.infiltration_column(t_end=2 * 3600.0)
    o = oracle_from_case(case)
    steps = o.run(case.t_end)
    mb = o.mass_balance()
    assert mb["closure_rel"] <= 1e-11
    assert mb["inflow_cum"] > 0 and mb["outflow_cum"] >= 0
    h, _ = o.get_state()
    assert h[-1] > -0.05 and h[0] <= -0.9     # wetted top, dry bottom after 2 h
    # the ponded front needs 10 EBATS reruns of the first step (1 s / 1.2^10)
    assert steps[0].rejected == 10 and steps[0].dt == pytest.approx(1.2 ** -10, rel=1e-12)
    assert all(s.picard <= 8 for s in steps)


def test_ponded_column_stalls_at_saturation_for_n_below_2():
    # For van Genuchten n < 2, dK/dh ~ (-alpha h)^(n-2) is unbounded as
    # h -> 0-, and with a ponded top the column approaches h = 0 under unit
    # gradient.  Classical Picard then cannot contract to 1e-6 m: EBATS
    # shrinks dt to dt_min and the step fails (documented finding; the same
    # column with n = 2 completes).
    case = W.infiltration_column(t_end=86400.0)
    o = oracle_from_case(case)
    with pytest.raises(O.OracleError, match="status 7"):
        o.run(case.t_end)
    _, meta = o.get_state()
    assert 7200.0 < meta["t"] < 9000.0


@pytest.mark.parametrize("nx,ny,dx,dy", [(3, 4, 0.02, 0.03), (5, 1, 0.5, 0.01), (1, 6, 0.01, 2.0)])
def test_laterally_uniform_block_equals_its_column(nx, ny, dx, dy):
    # With uniform soil, initial head and top/bottom conditions and zero-flux
    # sides, no lateral gradient ever forms: each column of the block follows
    # the 1 x 1 column exactly (lateral faces carry neither a pressure flux
    # nor gravity), per unit area, whatever the plan cell sizes.  Both solve
    # each linear system by the dense Cholesky factorisation, so the only
    # difference left is rounding.
    nz, dz = 24, 0.01
    bcs = [W.BC("zmax", "flux", np.array([0.0, 900.0]), np.array([5e-6, 0.0])), W.BC("zmin", "free_drainage")]
    params = dict(dt0=1.0, dt_max=120.0, solver=O.SOLVER_DENSE)
    col = oracle_from_case(_box(1, 1, nz, 1.0, 1.0, dz, [VG_SOIL], np.full(nz, -0.8), bcs, params))
    blk = oracle_from_case(_box(nx, ny, nz, dx, dy, dz, [VG_SOIL], np.full(nx * ny * nz, -0.8), bcs, params))
    sc, sb = col.run(1800.0), blk.run(1800.0)
    assert [(s.dt, s.picard, s.rejected) for s in sc] == [(s.dt, s.picard, s.rejected) for s in sb]
    hc, _ = col.get_state()
    hb, _ = blk.get_state()
    assert np.max(np.abs(hb.reshape(nz, ny, nx) - hc[:, None, None])) <= 1e-12
    mc, mb = col.mass_balance(), blk.mass_balance()
    area = nx * dx * ny * dy
    for k in ("storage", "inflow_cum", "outflow_cum"):
        assert mb[k] / area == pytest.approx(mc[k], rel=1e-12), k


def test_resume_from_a_saved_state_is_bit_identical():
    # set_state + set_clock (time, EBATS nominal step and easy-step counter)
    # resume a run exactly: the benchmark's CPU baseline starts the oracle
    # from a state saved by another run this way
    from paper_1809_10895_gb300 import workloads as W
    from tests.helpers import oracle_from_case
    case = W.heterogeneous_box(10, 8, 9, d=0.25, seed=4, water_table_depth=1.0, rain=6e-6, rain_hours=0.5)
    a = oracle_from_case(case)
    a.run(1500.0)
    h_mid, meta = a.get_state()
    rest_a = a.run(3000.0)
    b = oracle_from_case(case)
    b.set_state(h_mid, meta["t"])
    b.set_clock(meta["t"], meta["dt_nom"], meta["easy"])
    rest_b = b.run(3000.0)
    assert [(s.dt, s.picard, s.rejected) for s in rest_a] == [(s.dt, s.picard, s.rejected) for s in rest_b]
    assert np.array_equal(a.get_state()[0], b.get_state()[0])
    # the clock matters: without it EBATS restarts from dt0
    c = oracle_from_case(case)
    c.set_state(h_mid, meta["t"])
    assert [s.dt for s in c.run(3000.0)] != [s.dt for s in rest_a]
