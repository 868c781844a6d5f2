"""Pins of the oracle's modified Picard linearisation (Sec. 2.2: the
mass-conservative variant the paper implements beside the classical one; the
mixed form theta*(h^{k+1}) ~ theta*(h^k) + C(h^k)(h^{k+1} - h^k)).

Both linearisations have the same fixed point -- the backward-Euler step --
so from one state and one dt they must reach the same h^{n+1} within the
Picard tolerance; the modified form's storage term differs from the exact
change of water content only at second order in the last Picard update, so
its nonlinear mass defect is far below the chord form's; and it must reach
the closed-form steady profile of Appendix A (Eq. A8)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1809_10895_gb300 import workloads as W
from tests.golden.make_appendix_a import CONFIG, oracle_column
from tests.helpers import oracle_from_case

CASES = [lambda: W.infiltration_column(nz=60, dz=0.01, t_end=3600.0),
         lambda: W.heterogeneous_box(12, 10, 8, seed=3)]


def _state(case):
    o = oracle_from_case(case)
    o.run(600.0 if case.nx == 1 else 3600.0)
    return o.get_state()


@pytest.mark.parametrize("mk", CASES)
@pytest.mark.parametrize("dt", [1.0, 10.0, 60.0])
def test_same_backward_euler_step(mk, dt):
    case = mk()
    h0, meta = _state(case)
    out = {}
    for form in (0, 1):
        q = oracle_from_case(case, picard_form=form, dt0=dt, f_grow=1.0)
        q.set_state(h0, meta["t"])
        info = q.step()
        out[form] = (q.get_state()[0], info, q.mass_balance())
    # the same accepted dt (EBATS saw a converged attempt at the same dt) ...
    assert out[0][1].dt == out[1][1].dt
    # ... and the same step within the Picard tolerance (1e-6 m)
    assert np.max(np.abs(out[0][0] - out[1][0])) <= case.params["tol_picard"]
    for form in (0, 1):
        assert out[form][2]["closure_rel"] <= 1e-9


def test_modified_mass_defect_is_second_order():
    # one 10 s step of the column from a wetting state: the chord form's
    # defect is first order in the last Picard update, the modified form's
    # second order
    case = CASES[0]()
    h0, meta = _state(case)
    d = {}
    for form in (0, 1):
        q = oracle_from_case(case, picard_form=form, dt0=10.0, f_grow=1.0)
        q.set_state(h0, meta["t"])
        q.step()
        d[form] = abs(q.mass_balance()["nonlinear_defect_cum"])
    assert d[1] < 1e-2 * d[0]


def test_modified_run_conserves_mass():
    # half an hour of ponded infiltration with EBATS: both forms close the
    # balance of their linear systems; the modified form's accumulated
    # nonlinear defect is two orders below the chord form's
    case = CASES[0]()
    mb = {}
    for form in (0, 1):
        o = oracle_from_case(case, picard_form=form)
        o.run(1800.0)
        mb[form] = o.mass_balance()
        assert mb[form]["closure_rel"] <= 1e-9
    scale = mb[1]["storage0"] + mb[1]["inflow_cum"] + mb[1]["outflow_cum"]
    assert abs(mb[1]["nonlinear_defect_cum"]) <= 1e-10 * scale
    assert abs(mb[1]["nonlinear_defect_cum"]) <= 1e-2 * abs(mb[0]["nonlinear_defect_cum"])


def test_modified_reaches_appendix_a_profile():
    for q in (-1e-6, 9e-7):
        z, h = oracle_column(q, picard_form=1)
        exact = O.gardner_steady_profile(z, q, CONFIG["Ks"], CONFIG["alpha"])
        assert np.max(np.abs(h - exact)) <= 5e-5
