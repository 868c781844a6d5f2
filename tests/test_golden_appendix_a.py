"""Golden fixture: the steady Gardner column of Appendix A as printed (1 m,
100 cells of 1 cm, Ks = 1e-6 m/s, alpha = 0.06 1/m, water table at the
bottom, imposed top flux, PCG 1e-10, Picard 1e-8 m, dt 1 s .. 3600 s).
``tests/golden/appendix_a_gardner.json`` holds the oracle's profiles and the
closed form of Eq. A8 (written by ``tests/golden/make_appendix_a.py``)."""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from tests.golden.make_appendix_a import CONFIG, oracle_column

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "appendix_a_gardner.json")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def test_golden_matches_oracle_and_eq_a8():
    g = _golden()
    assert g["config"] == CONFIG
    for c in g["cases"]:
        z, h = oracle_column(c["q"])
        np.testing.assert_allclose(h, c["h_oracle"], rtol=0, atol=1e-12)
        exact = O.gardner_steady_profile(z, c["q"], CONFIG["Ks"], CONFIG["alpha"])
        np.testing.assert_allclose(exact, c["h_exact"], rtol=0, atol=1e-13)
        # the 1 cm discretisation of Eq. A8 (second order; see the oracle pins)
        assert np.max(np.abs(h - exact)) <= 5e-5


def test_golden_profiles_are_steady():
    cfg = dict(CONFIG, t_end=2 * CONFIG["t_end"])
    for c in _golden()["cases"]:
        _, h = oracle_column(c["q"], cfg)
        assert np.max(np.abs(h - np.array(c["h_oracle"]))) <= 1e-7


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-8), ("mixed", 1e-6)])
def test_gpu_reaches_the_golden_profiles(precision, tol):
    torch = pytest.importorskip("torch")
    from paper_1809_10895_gb300 import build, rf
    from paper_1809_10895_gb300 import workloads as W
    build.build()
    rf.load()
    torch.cuda.set_device(0)
    cfg = CONFIG
    nz = cfg["nz"]
    for c in _golden()["cases"]:
        soil = dict(model="gardner", theta_r=cfg["theta_r"], theta_s=cfg["theta_s"], alpha=cfg["alpha"],
                    Ks=cfg["Ks"], S=cfg["S"])
        case = W.Case(name="appendix_a", nx=1, ny=1, nz=nz, dx=1.0, dy=1.0, dz=cfg["L"] / nz, soils=[soil],
                      params=W.default_params(tol_cg=cfg["tol_cg"], tol_picard=cfg["tol_picard"], dt0=cfg["dt0"],
                                              dt_max=cfg["dt_max"]),
                      h0=-(np.arange(nz) + 0.5) * cfg["L"] / nz, t_end=cfg["t_end"])
        case.bcs = [W.BC("zmin", "dirichlet", np.array([0.0]), np.array([0.0])),
                    W.BC("zmax", "flux", np.array([0.0]), np.array([c["q"]]))]
        s = rf.Solver.from_case(case, precision=precision)
        s.run(cfg["t_end"])
        h = s.get_state()[0]
        assert np.max(np.abs(h - np.array(c["h_oracle"]))) <= tol, c["q"]
