"""GPU-vs-oracle parity through the C ABI.

Kernel level: closures + assembly, the stencil operator, one PCG solve.
Step level: per-step dt, Picard counts and rejections identical to the oracle,
max|h_gpu - h_oracle| <= 1e-8 m on the plain FP64 path (<= 1e-6 m on the mixed
path), global mass balance.  Inputs are seeded synthetic workloads at sizes
the oracle finishes in seconds (several thread blocks, ragged tails), plus the
full 128x128x64 box for its first steps.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1809_10895_gb300 import rf
from paper_1809_10895_gb300 import workloads as W
from tests.helpers import oracle_from_case

pytestmark = pytest.mark.gpu

TOL_PLAIN = 1e-8     # m, plain FP64 path vs oracle
TOL_MIXED = 1e-6     # m, FP32-inner defect-correction path vs oracle


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1809_10895_gb300 import build as B
    B.build()
    rf.load()
    torch.cuda.set_device(0)


def masked_case(nx=13, ny=7, nz=11, seed=4):
    """Masked, two-zone, heterogeneous grid with every boundary type."""
    rng = np.random.default_rng(seed)
    N = nx * ny * nz
    top = rng.integers(nz // 2, nz + 1, size=(ny, nx))
    k = np.arange(nz)[:, None, None]
    active = (k < top[None]).astype(np.uint8).ravel()
    soils = [dict(model="vg", theta_r=0.05, theta_s=0.40, alpha=2.0, n=1.8, Ks=1e-5, S=1e-5),
             dict(model="vg", theta_r=0.08, theta_s=0.45, alpha=2.3, n=1.2, Ks=1e-4, S=1e-4)]
    zone = (rng.random(N) < 0.4).astype(np.uint8)
    Ks = np.exp(np.log(1e-5) + rng.standard_normal(N))
    c = W.Case(name="masked", nx=nx, ny=ny, nz=nz, dx=0.3, dy=0.2, dz=0.1, z_bottom=-1.0, active=active,
               soils=soils, zone_of_cell=zone, Ks_cell=Ks, params=W.default_params(tol_cg=1e-13))
    c.bcs = [W.BC("zmin", "free_drainage"), W.BC("zmax", "flux", np.array([0.0, 50.0]), np.array([3e-6, 0.0])),
             W.BC("xmin", "dirichlet", np.array([0.0]), np.array([-0.4])),
             W.BC("ymax", "seepage")]
    h0 = -rng.uniform(0.01, 3.0, N)
    h0[rng.random(N) < 0.1] = rng.uniform(0.0, 0.3)
    c.h0 = h0
    return c


def gpu(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


# Relative error of theta* per closure arithmetic: FP64 (CUDA's log / exp
# against the oracle's pow, a few units in the last place: 1e-15); the
# double-float closures carry up to ~1.2e-14 (measured over alpha in
# [0.5, 5], n in [1.2, 2.6], h in [-1e3, -1e-6]), bounded by 3e-14.
THETA_REL = {"fp64": 1e-15, "double_float": 3e-14}


def chord_tol(case, hk, hn, dt, act, c_ref, arith="fp64"):
    """Bound on |c_gpu - c_oracle|: the chord slope divides a difference of
    theta values (<= 0.55) by h^k - h^n, so the theta error (two values) is
    amplified by 1/|h^k - h^n|; the rest is relative rounding."""
    V = case.dx * case.dy * case.dz
    dh = np.abs(hk - hn)[act]
    return (V / dt) * 2 * THETA_REL[arith] * 0.55 / np.maximum(dh, 1e-300) + 2e-12 * np.abs(c_ref)


@pytest.mark.parametrize("arith", ["fp64", "double_float"])
def test_assembly_matches_oracle(arith):
    case = masked_case()
    o = oracle_from_case(case)
    s = rf.Solver.from_case(case, closure_arith=arith)
    rng = np.random.default_rng(9)
    hk = case.h0 + rng.normal(0, 0.05, case.N)
    out = {k: torch.zeros(case.N, dtype=torch.float64, device="cuda") for k in ("K", "theta", "c", "b", "diag")}
    for t in (0.0, 60.0):          # before and after the flux breakpoint
        s.assemble(gpu(hk), gpu(case.h0), 37.0, t, **out)
        ref = o.assemble(hk, case.h0, 37.0, t)
        act = o.active_cells
        # K: the oracle's literal Eq. 4 loses digits to cancellation in wet
        # soil (1 - Se^(1/m)); theta*: the closure arithmetic's own bound
        np.testing.assert_allclose(out["K"].cpu().numpy()[act], ref["K"], rtol=2e-12, atol=0, err_msg="K")
        np.testing.assert_allclose(out["theta"].cpu().numpy()[act], ref["theta"], rtol=THETA_REL[arith], atol=0,
                                   err_msg="theta")
        tol_c = chord_tol(case, hk, case.h0, 37.0, act, ref["c"], arith)
        assert np.all(np.abs(out["c"].cpu().numpy()[act] - ref["c"]) <= tol_c)
        assert np.all(np.abs(out["diag"].cpu().numpy()[act] - ref["diag"]) <= tol_c + 2e-12 * ref["diag"])
        bg = out["b"].cpu().numpy()[act]
        # b = c h^n + gravity + boundary terms inherits the chord error of c
        tol_b = tol_c * np.abs(case.h0[act]) + 1e-11 * np.abs(ref["b"]) + 1e-14 * np.abs(ref["b"]).max()
        assert np.all(np.abs(bg - ref["b"]) <= tol_b)
        inact = np.setdiff1d(np.arange(case.N), act)
        assert np.all(out["diag"].cpu().numpy()[inact] == 0)


def test_operator_and_solve_match_oracle():
    case = masked_case(17, 9, 13, seed=5)
    o = oracle_from_case(case)
    s = rf.Solver.from_case(case)
    rng = np.random.default_rng(2)
    hk = case.h0 + rng.normal(0, 0.02, case.N)
    s.assemble(gpu(hk), gpu(case.h0), 120.0, 0.0)
    act = o.active_cells
    xfull = np.zeros(case.N)
    xfull[act] = rng.standard_normal(len(act))
    y = torch.zeros(case.N, dtype=torch.float64, device="cuda")
    s.apply(gpu(xfull), y)
    yo = o.spmv(hk, case.h0, 120.0, xfull[act])
    # (A x)_P differs by the chord error of c_P times |x_P| plus rounding of
    # terms of size diag |x|
    ref = o.assemble(hk, case.h0, 120.0)
    tol = chord_tol(case, hk, case.h0, 120.0, act, ref["c"]) * np.abs(xfull[act]) \
        + 1e-14 * ref["diag"].max() * np.abs(xfull).max()
    assert np.all(np.abs(y.cpu().numpy()[act] - yo) <= tol)
    # one PCG solve from x0 = h^k
    x = gpu(hk)
    it = s.solve(x)
    xo, ito, _ = o.solve(hk, case.h0, 120.0)
    assert abs(it - ito) <= 1
    # the two systems differ by the chord error of c (above, FP64 closures);
    # the solutions agree to 1e-10 m, two orders below the step-level 1e-8 m
    assert np.max(np.abs(x.cpu().numpy()[act] - xo)) <= 1e-10


def _run_pair(case, t_end, **over):
    s = rf.Solver.from_case(case, **over)
    o = oracle_from_case(case, **{k: v for k, v in over.items()
                                  if k not in ("precision", "tol_inner", "closure_arith", "precond")})
    sg = s.run(t_end)
    so = o.run(t_end)
    return s, o, sg, so


def _assert_same_sequence(sg, so):
    assert len(sg) == len(so)
    dts = np.array([[a.dt, b.dt] for a, b in zip(sg, so)])
    assert np.array_equal(dts[:, 0], dts[:, 1])
    assert [a.picard for a in sg] == [b.picard for b in so]
    assert [a.rejected for a in sg] == [b.rejected for b in so]


def test_infiltration_column_first_two_hours():
    case = W.infiltration_column(t_end=2 * 3600.0)
    s, o, sg, so = _run_pair(case, case.t_end)
    _assert_same_sequence(sg, so)
    hg, mg = s.get_state()
    ho, mo = o.get_state()
    assert np.max(np.abs(hg - ho)) <= TOL_PLAIN
    assert mg["t"] == mo["t"] and mg["dt_nom"] == mo["dt_nom"]
    mbg, mbo = s.mass_balance(), o.mass_balance()
    assert mbg["closure_rel"] <= 1e-11
    assert mbg["inflow_cum"] == pytest.approx(mbo["inflow_cum"], rel=1e-9)


def test_heterogeneous_box_parity():
    case = W.heterogeneous_box(21, 13, 17, d=0.25, seed=7, water_table_depth=2.0, rain=4e-6, rain_hours=1.0,
                               t_end=4 * 3600.0)
    s, o, sg, so = _run_pair(case, case.t_end)
    _assert_same_sequence(sg, so)
    hg, _ = s.get_state()
    ho, _ = o.get_state()
    assert np.max(np.abs(hg - ho)) <= TOL_PLAIN
    mbg, mbo = s.mass_balance(), o.mass_balance()
    # boundary fluxes at a hydrostatic Dirichlet face nearly cancel, so they
    # are compared against the stored volume, not their own size
    for k in ("storage", "inflow_cum", "outflow_cum"):
        assert abs(mbg[k] - mbo[k]) <= 1e-12 * mbo["storage0"]
    # the linear closure is sum dt (A x - b), bounded by the CG tolerance
    assert mbg["closure_rel"] <= 1e-9
    assert mbg["closure_rel"] <= 10 * mbo["closure_rel"] + 1e-12


def test_masked_watershed_parity():
    # seed 0 rains from hour 11 (3.4 mm/h, 11.4 mm/h from hour 17)
    case = W.watershed(24, 20, 16, dx=10.0, dz=0.5, seed=0, hours=24, tol_cg=1e-12)
    s, o, sg, so = _run_pair(case, 20 * 3600.0)
    assert s.mass_balance()["inflow_cum"] > 0.0
    _assert_same_sequence(sg, so)
    hg, _ = s.get_state()
    ho, _ = o.get_state()
    act = case.active.astype(bool)
    assert np.max(np.abs(hg - ho)[act]) <= TOL_PLAIN


def test_mixed_precision_path():
    case = W.heterogeneous_box(21, 13, 17, d=0.25, seed=7, water_table_depth=2.0, rain=4e-6, rain_hours=1.0,
                               t_end=4 * 3600.0)
    s = rf.Solver.from_case(case, precision="mixed")
    o = oracle_from_case(case)
    s.run(case.t_end)
    o.run(case.t_end)
    hg, _ = s.get_state()
    ho, _ = o.get_state()
    assert np.max(np.abs(hg - ho)) <= TOL_MIXED
    mb = s.mass_balance()
    assert mb["closure_rel"] <= 1e-9


def test_runs_are_bit_reproducible():
    case = W.heterogeneous_box(19, 11, 9, d=0.25, seed=8, water_table_depth=1.0, rain=8e-6)
    outs = []
    for _ in range(2):
        s = rf.Solver.from_case(case)
        s.run(900.0)
        outs.append(s.get_state()[0])
    assert np.array_equal(outs[0], outs[1])


def test_checkpoint_resume_is_bit_identical():
    case = W.heterogeneous_box(10, 9, 12, d=0.25, seed=1, water_table_depth=1.0, t_end=1800.0)
    a = rf.Solver.from_case(case)
    a.run(900.0)
    h_mid, meta = a.get_state()
    mb = a.mass_balance()
    a.run(1800.0)
    b = rf.Solver.from_case(case)
    b.set_state(h_mid, meta["t"])
    mass7 = [mb["storage0"], 0.0, mb["inflow_cum"], mb["outflow_cum"], 0.0, 0.0, mb["nonlinear_defect_cum"]]
    b.set_meta(meta, mass7)
    b.run(1800.0)
    assert np.array_equal(a.get_state()[0], b.get_state()[0])
    # the state read into a caller's pinned buffer is the same
    pinned = torch.empty(case.N, dtype=torch.float64, pin_memory=True).numpy()
    h, meta_b = b.get_state(out=pinned)
    assert h is pinned and np.array_equal(pinned, a.get_state()[0]) and meta_b["t"] == a.get_state()[1]["t"]
    with pytest.raises(ValueError):
        b.get_state(out=np.empty(case.N, dtype=np.float32))


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 2), (3, 1, 1), (2, 3, 1), (1, 5, 7), (33, 1, 9)])
def test_tiny_and_degenerate_grids(shape):
    nx, ny, nz = shape
    case = W.Case(name="tiny", nx=nx, ny=ny, nz=nz, dx=0.1, dy=0.1, dz=0.05,
                  soils=[dict(model="vg", theta_r=0.05, theta_s=0.4, alpha=2.0, n=1.8, Ks=1e-5, S=1e-5)],
                  params=W.default_params(tol_cg=1e-13))
    case.h0 = np.linspace(-1.0, -0.2, case.N)
    case.bcs = [W.BC("zmax", "flux", np.array([0.0]), np.array([2e-6])), W.BC("zmin", "free_drainage")]
    s, o, sg, so = _run_pair(case, 600.0)
    _assert_same_sequence(sg, so)
    assert np.max(np.abs(s.get_state()[0] - o.get_state()[0])) <= TOL_PLAIN


def test_all_inactive_columns_and_hydrostatic_fixed_point():
    nx, ny, nz = 6, 5, 8
    active = np.ones(nx * ny * nz, dtype=np.uint8)
    active.reshape(nz, ny, nx)[:, 2, 3] = 0          # a fully inactive column
    active.reshape(nz, ny, nx)[5:, 0, :] = 0         # a terrace
    case = W.Case(name="hydro", nx=nx, ny=ny, nz=nz, dx=0.2, dy=0.2, dz=0.25, active=active,
                  soils=[dict(model="vg", theta_r=0.05, theta_s=0.4, alpha=2.0, n=1.8, Ks=1e-5, S=1e-5)],
                  params=W.default_params(tol_cg=1e-13))
    case.h0 = 1.0 - case.z_centres()
    case.bcs = [W.BC("zmin", "dirichlet", np.array([0.0]), np.array([1.0]))]
    s = rf.Solver.from_case(case)
    steps = s.run(3600.0)
    assert all(x.picard == 1 for x in steps)
    h, _ = s.get_state()
    act = active.astype(bool)
    assert np.max(np.abs(h - case.h0)[act]) <= 1e-12


def test_error_paths():
    case = masked_case()
    s = rf.Solver(case.nx, case.ny, case.nz, case.dx, case.dy, case.dz)
    with pytest.raises(rf.RFError) as e:
        s.step()
    assert e.value.status == rf.RF_ERR_STATE
    with pytest.raises(rf.RFError) as e:
        s.set_bc("xmin", "free_drainage")
    assert e.value.status == rf.RF_ERR_ARG
    with pytest.raises(rf.RFError) as e:
        s.set_soils([dict(model="vg", theta_r=0.05, theta_s=0.4, alpha=2.0, n=0.9, Ks=1e-5)])
    assert e.value.status == rf.RF_ERR_ARG
    with pytest.raises(rf.RFError) as e:
        s.set_params(f_shrink=1.0)
    assert e.value.status == rf.RF_ERR_ARG


def test_state_set_checks_heads_on_the_device():
    # a non-finite head on an active cell is refused (RF_ERR_ARG) and leaves
    # the state and clock as they were; non-finite values on inactive cells
    # are accepted and stored as 0
    case = W.watershed(24, 20, 16, dx=10.0, dz=0.5, seed=0, hours=24, tol_cg=1e-12)
    s = rf.Solver.from_case(case)
    s.run(600.0)
    h0, m0 = s.get_state()
    act = case.active.astype(bool)
    bad = h0.copy()
    bad[np.flatnonzero(act)[7]] = np.nan
    with pytest.raises(rf.RFError) as e:
        s.set_state(bad, 0.0)
    assert e.value.status == rf.RF_ERR_ARG
    h1, m1 = s.get_state()
    assert np.array_equal(h0, h1) and m0 == m1
    ok = h0.copy()
    ok[np.flatnonzero(~act)[:5]] = np.inf
    s.set_state(ok, 5.0)
    h2, m2 = s.get_state()
    assert np.array_equal(h2[act], h0[act]) and np.all(h2[np.flatnonzero(~act)[:5]] == 0.0) and m2["t"] == 5.0


def test_dt_min_failure_leaves_state_unchanged():
    # one Picard iteration allowed and an unreachable tolerance: every try is
    # rejected, EBATS shrinks dt below dt_min and the call fails with
    # RF_ERR_DT_MIN, state and EBATS counters untouched
    case = W.heterogeneous_box(8, 8, 10, d=0.25, seed=2, water_table_depth=1.0, rain=1e-5)
    s = rf.Solver.from_case(case, tol_picard=1e-30, n_max=1, dt_min=0.2)
    h0, m0 = s.get_state()
    with pytest.raises(rf.RFError) as e:
        s.step()
    assert e.value.status == rf.RF_ERR_DT_MIN
    h1, m1 = s.get_state()
    assert np.array_equal(h0, h1) and m0 == m1


@pytest.mark.parametrize("precision,tol", [("fp64", TOL_PLAIN), ("mixed", TOL_MIXED)])
def test_full_size_box_first_steps(precision, tol):
    # the 128x128x64 heterogeneous box at full size (the mixed path runs the
    # TMA-staged FP32 stencil over two x-tiles): first steps vs oracle
    case = W.heterogeneous_box(seed=0)
    s = rf.Solver.from_case(case, precision=precision)
    o = oracle_from_case(case)
    for _ in range(3):
        a, b = s.step(), o.step()
        assert (a.dt, a.picard, a.rejected) == (b.dt, b.picard, b.rejected)
    assert np.max(np.abs(s.get_state()[0] - o.get_state()[0])) <= tol


# Grids that take the mixed path's TMA-staged FP32 stencil (nx a multiple of
# 4) across 128-cell x-tiles with a ragged last tile, all active and masked,
# and one that takes the plain-tile FP32 stencil (nx odd).
def _box_multitile():
    return W.heterogeneous_box(136, 20, 12, d=0.25, seed=21, water_table_depth=2.0, rain=4e-6, rain_hours=1.0,
                               t_end=2 * 3600.0)


def _watershed_multitile():
    # seed 0 rains from hour 11 (3.4 mm/h, 11.4 mm/h from hour 17)
    return W.watershed(132, 24, 16, dx=10.0, dz=0.5, seed=0, hours=24, tol_cg=1e-12)


def _box_wide():
    # three x-tiles of the TMA stencil, the last one 8 cells wide
    return W.heterogeneous_box(264, 12, 6, d=0.25, seed=23, water_table_depth=1.0, rain=4e-6, rain_hours=1.0,
                               t_end=3600.0)


def _box_odd():
    return W.heterogeneous_box(135, 21, 11, d=0.25, seed=22, water_table_depth=2.0, rain=4e-6, rain_hours=1.0,
                               t_end=2 * 3600.0)


@pytest.mark.parametrize("make,t_end", [(_box_multitile, 2 * 3600.0), (_watershed_multitile, 20 * 3600.0),
                                        (_box_odd, 2 * 3600.0)], ids=["box136x20x12", "watershed132x24x16",
                                                                      "box135x21x11"])
def test_mixed_path_multitile_parity(make, t_end):
    case = make()
    s, o, sg, so = _run_pair(case, t_end, precision="mixed")
    _assert_same_sequence(sg, so)
    hg, _ = s.get_state()
    ho, _ = o.get_state()
    act = np.ones(case.N, bool) if case.active is None else case.active.astype(bool)
    assert np.max(np.abs(hg - ho)[act]) <= TOL_MIXED
    assert s.mass_balance()["closure_rel"] <= 1e-9


def _inner_operator_bound(case, o, hk, hn, dt, p64, act):
    """Element-wise bound on |q32 - A p| for the FP32 operator: FP32 rounding
    of K, cb and w (one unit each) and of the products and sums that form q
    (about ten per face), u = 2^-24 relative to the sum of term magnitudes,
    plus the FP64 chord difference of c between the two sides times |p|."""
    ref = o.assemble(hk, hn, dt)
    absq = o.spmv(hk, hn, dt, np.abs(p64[act]))          # diag |p| - sum T |p_N| <= sum of magnitudes
    # sum of term magnitudes = diag |p_P| + sum_f T_f |p_N| = 2 diag |p| - (A |p|)
    mags = 2 * ref["diag"] * np.abs(p64[act]) - absq
    u = 2.0 ** -24
    return 16 * u * mags + chord_tol(case, hk, hn, dt, act, ref["c"]) * np.abs(p64[act])


@pytest.mark.parametrize("make", [_box_multitile, _watershed_multitile, _box_wide, _box_odd],
                         ids=["box136x20x12", "watershed132x24x16", "box264x12x6", "box135x21x11"])
def test_inner_fp32_operator_matches_oracle(make):
    case = make()
    o = oracle_from_case(case)
    s = rf.Solver.from_case(case, precision="mixed")
    rng = np.random.default_rng(31)
    hk = case.h0 + rng.normal(0, 0.02, case.N)
    s.assemble(gpu(hk), gpu(case.h0), 90.0, 0.0)
    act_mask = np.ones(case.N, bool) if case.active is None else case.active.astype(bool)
    act = o.active_cells
    f32 = dict(dtype=torch.float32, device="cuda")
    z = rng.standard_normal(case.N).astype(np.float32)
    pold = rng.standard_normal(case.N).astype(np.float32)
    for beta in (0.0, 0.37):
        p = torch.zeros(case.N, **f32)
        q = torch.zeros(case.N, **f32)
        pq = s.apply_inner(torch.as_tensor(z, **f32), p, q, pold=torch.as_tensor(pold, **f32), beta=beta)
        pg, qg = p.cpu().numpy().astype(np.float64), q.cpu().numpy().astype(np.float64)
        # p = fma(beta, p_old, z) in FP32 with beta an FP32 value: the exact
        # value rounded once (half a unit), 0 off the active set
        b32 = float(np.float32(beta))
        pr = z.astype(np.float64) + b32 * pold.astype(np.float64)
        mag = np.abs(z.astype(np.float64)) + np.abs(b32 * pold.astype(np.float64))
        assert np.all(np.abs(pg - pr)[act_mask] <= 2.0 ** -24 * np.abs(pr[act_mask]) + 2.0 ** -50 * mag[act_mask])
        assert np.all(pg[~act_mask] == 0) and np.all(qg[~act_mask] == 0)
        # q = A p element by element against the oracle's CSR operator on the same p
        qo = o.spmv(hk, case.h0, 90.0, pg[act])
        tol = _inner_operator_bound(case, o, hk, case.h0, 90.0, pg, act)
        err = np.abs(qg[act] - qo)
        assert np.all(err <= tol), (beta, float(np.max(err / tol)))
        assert pq == pytest.approx(float(pg[act] @ qo), rel=1e-5)


def test_device_wait_timeout_is_reported_and_the_context_recovers():
    # a wait for staged stencil data that gives up at its first test stops
    # the solve; the copies in flight are drained with the normal limit, the
    # step returns RF_ERR_DEVICE_TIMEOUT with the state unchanged, and the
    # same context then steps exactly like the oracle
    case = _box_multitile()
    s = rf.Solver.from_case(case, precision="mixed")
    h0, m0 = s.get_state()
    s.set_wait_limit(-1)
    with pytest.raises(rf.RFError) as e:
        s.step()
    assert e.value.status == rf.RF_ERR_DEVICE_TIMEOUT
    h1, m1 = s.get_state()
    assert np.array_equal(h0, h1) and m0 == m1
    s.set_wait_limit(0)
    o = oracle_from_case(case)
    for _ in range(6):
        a, b = s.step(), o.step()
        assert (a.dt, a.picard, a.rejected) == (b.dt, b.picard, b.rejected)
    assert np.max(np.abs(s.get_state()[0] - o.get_state()[0])) <= TOL_MIXED
