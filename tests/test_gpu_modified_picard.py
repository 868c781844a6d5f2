"""Modified Picard (Sec. 2.2's mass-conservative linearisation) on the GPU
against the oracle's modified Picard: identical dt / Picard / rejection
sequences, max|h_gpu - h_oracle| <= 1e-8 m (plain FP64) or 1e-6 m (mixed),
water balance; the same backward-Euler step as the classical (chord) form
from one state; switching the form on a live solver; the batched ensemble
refuses it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1809_10895_gb300 import rf
from paper_1809_10895_gb300 import workloads as W
from tests.helpers import oracle_from_case
from tests.test_gpu_parity import TOL_MIXED, TOL_PLAIN, _assert_same_sequence, _run_pair

pytestmark = pytest.mark.gpu

MOD = dict(picard_form=1)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1809_10895_gb300 import build as B
    B.build()
    rf.load()
    torch.cuda.set_device(0)


def test_column_modified_matches_oracle():
    case = W.infiltration_column(nz=60, dz=0.01, t_end=1800.0)
    s, o, sg, so = _run_pair(case, case.t_end, **MOD)
    _assert_same_sequence(sg, so)
    assert np.max(np.abs(s.get_state()[0] - o.get_state()[0])) <= TOL_PLAIN
    mbg, mbo = s.mass_balance(), o.mass_balance()
    assert mbg["closure_rel"] <= 1e-11
    assert mbg["inflow_cum"] == pytest.approx(mbo["inflow_cum"], rel=1e-9)
    scale = mbg["storage0"] + mbg["inflow_cum"] + mbg["outflow_cum"]
    assert abs(mbg["nonlinear_defect_cum"]) <= 1e-10 * scale


def test_box_and_masked_modified_match_oracle():
    box = W.heterogeneous_box(21, 13, 17, d=0.25, seed=7, water_table_depth=2.0, rain=4e-6, rain_hours=1.0,
                              t_end=4 * 3600.0)
    ws = W.watershed(24, 20, 16, dx=10.0, dz=0.5, seed=3, hours=24, tol_cg=1e-12)   # masked terrain
    for case, t_end in ((box, box.t_end), (ws, 12 * 3600.0)):
        s, o, sg, so = _run_pair(case, t_end, **MOD)
        _assert_same_sequence(sg, so)
        act = np.asarray(case.active, bool) if case.active is not None else slice(None)
        assert np.max(np.abs(s.get_state()[0] - o.get_state()[0])[act]) <= TOL_PLAIN
        assert s.mass_balance()["closure_rel"] <= 1e-9


def test_mixed_modified_matches_oracle():
    case = W.heterogeneous_box(21, 13, 17, d=0.25, seed=7, water_table_depth=2.0, rain=4e-6, rain_hours=1.0,
                               t_end=4 * 3600.0)
    s = rf.Solver.from_case(case, precision="mixed", picard_form="modified")
    o = oracle_from_case(case, **MOD)
    s.run(case.t_end)
    o.run(case.t_end)
    assert np.max(np.abs(s.get_state()[0] - o.get_state()[0])) <= TOL_MIXED
    assert s.mass_balance()["closure_rel"] <= 1e-9


def test_same_step_as_chord_and_live_switch():
    case = W.infiltration_column(nz=60, dz=0.01, t_end=3600.0)
    s = rf.Solver.from_case(case)
    s.run(600.0)
    h0, meta = s.get_state()
    out = {}
    for form in ("chord", "modified"):
        s.set_params(picard_form=form, dt0=10.0, f_grow=1.0)   # switches a live solver
        s.set_state(h0, meta["t"])                              # dt_nom <- dt0
        info = s.step()
        out[form] = (s.get_state()[0], info)
    assert out["chord"][1].dt == out["modified"][1].dt
    assert np.max(np.abs(out["chord"][0] - out["modified"][0])) <= case.params["tol_picard"]


def test_ensemble_refuses_modified_picard():
    cases = W.ensemble(2, seed=1, t_end=60.0, max_side=2, nz_range=(10, 12))
    with pytest.raises(RuntimeError):
        rf.Ensemble.from_cases(cases, picard_form="modified")
