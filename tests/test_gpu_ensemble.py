"""Batched ensemble (one persistent graph-launched kernel) against the CPU
oracle run instance by instance: identical step / Picard / rejection totals,
heads within 1e-8 m (FP64) or 1e-6 m (mixed), for single-CTA and multi-CTA
cluster work units, every CTA size, and clusters that hand the smaller
instances to single CTAs; the vertical-line preconditioner on the same
tilings, and its exactness on vertical flow; laterally uniform instances
equal their 1x1 column; the tuner picks a working tile."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1809_10895_gb300 import rf
from paper_1809_10895_gb300 import workloads as W
from tests.helpers import oracle_from_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1809_10895_gb300 import build as B
    B.build()
    rf.load()
    torch.cuda.set_device(0)


def small_ensemble(n=7, seed=3):
    return W.ensemble(n, seed=seed, t_end=1800.0, max_side=4, nz_range=(20, 60))


@pytest.fixture(scope="module")
def oracle_runs():
    cases = small_ensemble()
    out = []
    for c in cases:
        o = oracle_from_case(c)
        steps = o.run(c.t_end)
        h, _ = o.get_state()
        out.append((h, steps, o.mass_balance()))
    return cases, out


@pytest.mark.parametrize("cluster,threads,wide", [(1, 512, 0), (4, 512, 0), (1, 128, 0), (2, 256, 0), (4, 128, 1),
                                                  (8, 256, 2)])
def test_ensemble_fp64_matches_oracle(oracle_runs, cluster, threads, wide):
    cases, ref = oracle_runs
    e = rf.Ensemble.from_cases(cases, precision="fp64")
    e.set_tiling(cluster, threads)
    # wide k: the first k instances of a reversed order on whole clusters, the
    # rest on single CTAs
    order = list(range(len(cases)))[::-1]
    if wide:
        e.set_schedule(order, wide)
    e.run(cases[0].t_end)
    for i, (c, (ho, so, mbo)) in enumerate(zip(cases, ref)):
        h, st = e.get(i)
        assert st["status"] == 0 and st["t"] == pytest.approx(c.t_end, abs=1e-6)
        assert st["ctas"] == (cluster if not wide or order.index(i) < wide else 1)
        assert st["busy_s"] > 0
        assert st["steps"] == len(so)
        assert st["picard_iters"] == sum(s.picard for s in so)
        assert st["rejected"] == sum(s.rejected for s in so)
        assert np.max(np.abs(h - ho)) <= 1e-8, i
        assert st["inflow_cum"] == pytest.approx(mbo["inflow_cum"], rel=1e-8)
        # the linear closure is set by the CG tolerance: compare with the
        # oracle's own closure on the same instance
        scale = st["storage0"] + st["inflow_cum"] + st["outflow_cum"]
        assert st["closure_abs"] / scale <= 10 * mbo["closure_rel"] + 1e-12


def test_ensemble_mixed_matches_oracle(oracle_runs):
    cases, ref = oracle_runs
    e = rf.Ensemble.from_cases(cases, precision="mixed")
    e.set_tiling(2, 128)
    e.run(cases[0].t_end)
    for i, (c, (ho, so, mbo)) in enumerate(zip(cases, ref)):
        h, st = e.get(i)
        assert st["status"] == 0
        assert np.max(np.abs(h - ho)) <= 1e-6, i
        scale = st["storage0"] + st["inflow_cum"] + st["outflow_cum"]
        assert st["closure_abs"] / scale <= 10 * mbo["closure_rel"] + 1e-12


@pytest.mark.parametrize("cluster,threads,wide", [(1, 512, 0), (4, 128, 0), (8, 256, 2)])
def test_ensemble_vertical_line_preconditioner_matches_oracle(oracle_runs, cluster, threads, wide):
    """Mixed path with the vertical-line preconditioner: same heads as the
    oracle within the mixed path's 1e-6 m, on single CTAs and on clusters
    whose CTAs' cell ranges cut every column (the columns' solves read and
    write across the CTAs)."""
    cases, ref = oracle_runs
    e = rf.Ensemble.from_cases(cases, precision="mixed", precond="zline")
    e.set_tiling(cluster, threads)
    if wide:
        e.set_schedule(None, wide)
    e.run(cases[0].t_end)
    for i, (c, (ho, so, mbo)) in enumerate(zip(cases, ref)):
        h, st = e.get(i)
        assert st["status"] == 0 and st["t"] == pytest.approx(c.t_end, abs=1e-6)
        assert np.max(np.abs(h - ho)) <= 1e-6, i
        scale = st["storage0"] + st["inflow_cum"] + st["outflow_cum"]
        assert st["closure_abs"] / scale <= 10 * mbo["closure_rel"] + 1e-12


def test_vertical_line_preconditioner_is_exact_on_vertical_flow():
    """On 1x1 columns and on laterally uniform blocks the line solve is the
    inverse of the operator (no horizontal flux), so each inner PCG ends
    after one iteration (to FP32 rounding, far below the inner tolerance
    1e-4): inner iterations = defect-correction passes, two or three per
    Picard iteration at the outer tolerance 1e-10, where Jacobi needs
    several times more on 1 cm cells."""
    base = small_ensemble(3, seed=5)
    cases = []
    for c in base:
        for nx, ny in ((1, 1), (3, 2)):
            cases.append(W.Case(name=f"{c.name}_{nx}x{ny}", nx=nx, ny=ny, nz=c.nz, dx=c.dx, dy=c.dy, dz=c.dz,
                                soils=c.soils, bcs=c.bcs, params=c.params,
                                h0=np.full(nx * ny * c.nz, c.h0[0]), t_end=c.t_end))
    runs = {}
    for pc in ("jacobi", "zline"):
        e = rf.Ensemble.from_cases(cases, precision="mixed", precond=pc)
        e.set_tiling(2, 128)
        e.run(cases[0].t_end)
        runs[pc] = [e.get(i) for i in range(len(cases))]
    tot = {pc: [sum(st[k] for _, st in runs[pc]) for k in ("cg_iters", "picard_iters")] for pc in runs}
    for i, c in enumerate(cases):
        (hj, sj), (hz, sz) = runs["jacobi"][i], runs["zline"][i]
        assert sz["status"] == 0 and sj["status"] == 0
        assert sz["cg_iters"] <= 4 * sz["picard_iters"], c.name
        assert np.max(np.abs(hz - hj)) <= 2e-6, c.name
    assert tot["zline"][0] <= 3 * tot["zline"][1]
    assert tot["jacobi"][0] >= 2 * tot["zline"][0]


def test_laterally_uniform_instance_equals_its_column():
    base = small_ensemble(1, seed=9)[0]
    col = W.Case(name="col", nx=1, ny=1, nz=base.nz, dx=base.dx, dy=base.dy, dz=base.dz, soils=base.soils,
                 bcs=base.bcs, params=base.params, h0=np.full(base.nz, base.h0[0]), t_end=base.t_end)
    blk = W.Case(name="blk", nx=3, ny=2, nz=base.nz, dx=base.dx, dy=base.dy, dz=base.dz, soils=base.soils,
                 bcs=base.bcs, params=base.params, h0=np.full(6 * base.nz, base.h0[0]), t_end=base.t_end)
    e = rf.Ensemble.from_cases([col, blk], precision="fp64")
    e.run(base.t_end)
    hc, sc = e.get(0)
    hb, sb = e.get(1)
    assert (sc["steps"], sc["picard_iters"]) == (sb["steps"], sb["picard_iters"])
    hb2 = hb.reshape(base.nz, 6)
    # the block stays laterally uniform up to rounding (edge and interior
    # columns round their zero lateral fluxes differently, and the linear
    # solves amplify that over ~10^3 solves) ...
    assert np.max(hb2.max(1) - hb2.min(1)) <= 1e-10
    # ... and equals the column up to where the relative CG stop lands
    # (the block's ||b|| is sqrt(6) times the column's)
    assert np.max(np.abs(hb2 - hc[:, None])) <= 1e-8


def test_tuner_picks_a_working_tile(oracle_runs):
    cases, ref = oracle_runs
    e = rf.Ensemble.from_cases(cases, precision="fp64")
    cl, th, wide, ms = e.tune(300.0)
    assert cl in (1, 2, 4, 8) and th in (256, 512) and wide == len(cases) and ms > 0
    e.run(cases[0].t_end)
    for i, (ho, so, _) in enumerate(ref):
        h, st = e.get(i)
        assert st["steps"] == len(so)
        assert np.max(np.abs(h - ho)) <= 1e-8
