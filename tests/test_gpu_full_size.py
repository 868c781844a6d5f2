"""Full-size configurations, in the launch configuration the benchmark times:
the 512x512x64 watershed (sampled assembly outputs against the oracle, water
balance), the 256-instance uneven ensemble (sampled instances against the
oracle run one by one, every instance's balance) and a warm-started step on
a 512x512x64 box (against the plain step of the same size)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1809_10895_gb300 import rf, warmstart
from paper_1809_10895_gb300 import workloads as W
from tests.helpers import oracle_from_case
from tests.test_gpu_parity import chord_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1809_10895_gb300 import build as B
    B.build()
    rf.load()
    torch.cuda.set_device(0)


def gpu(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("precond", ["jacobi", "mg"])
def test_watershed_full_size(precond):
    case = W.watershed(512, 512, 64, seed=0, hours=24)
    s = rf.Solver.from_case(case, precision="mixed", precond=precond)
    infos = [s.step() for _ in range(3)]
    h, meta = s.get_state()
    act = np.asarray(case.active, bool)
    assert np.all(np.isfinite(h[act]))
    assert all(i.rejected == 0 for i in infos)
    mb = s.mass_balance()
    assert mb["closure_rel"] <= 1e-9
    if precond == "mg":
        return
    # the system at the reached state, sampled cells against the oracle
    o = oracle_from_case(case)
    dt, t = 600.0, meta["t"]
    out = {k: torch.zeros(case.N, dtype=torch.float64, device="cuda") for k in ("K", "theta", "c", "b", "diag")}
    s.assemble(gpu(h), gpu(case.h0), dt, t, **out)
    ref = o.assemble(h, case.h0, dt, t)
    ia = o.active_cells                                   # active cell indices, oracle order
    pick = np.random.default_rng(1).choice(len(ia), size=20000, replace=False)
    cells = ia[pick]
    for key in ("K", "theta"):
        np.testing.assert_allclose(out[key].cpu().numpy()[cells], ref[key][pick], rtol=2e-12, atol=0, err_msg=key)
    tol_c = chord_tol(case, h, case.h0, dt, cells, ref["c"][pick])
    assert np.all(np.abs(out["c"].cpu().numpy()[cells] - ref["c"][pick]) <= tol_c)
    assert np.all(np.abs(out["diag"].cpu().numpy()[cells] - ref["diag"][pick]) <= tol_c + 2e-12 * ref["diag"][pick])
    bg, br = out["b"].cpu().numpy()[cells], ref["b"][pick]
    tol_b = tol_c * np.abs(case.h0[cells]) + 1e-11 * np.abs(br) + 1e-14 * np.abs(ref["b"]).max()
    assert np.all(np.abs(bg - br) <= tol_b)


@pytest.mark.parametrize("precond,tiling", [("jacobi", None), ("zline", (8, 256))])
def test_ensemble_full_size(precond, tiling):
    """The 256-instance workload (the bench's ensemble: vertical-line
    preconditioner on 8-CTA clusters of 256 threads) over its first minute:
    every instance's balance closes; the two smallest and two largest
    instances match the oracle."""
    cases = W.ensemble(256, seed=0)
    window = 60.0
    e = rf.Ensemble.from_cases(cases, precision="mixed", precond=precond)
    if tiling:
        e.set_tiling(*tiling)
    e.run(window)
    stats = [e.get(i, want_h=False)[1] for i in range(len(cases))]
    for st in stats:
        assert st["status"] == 0 and st["t"] == pytest.approx(window, abs=1e-6)
        scale = st["storage0"] + st["inflow_cum"] + st["outflow_cum"]
        assert st["closure_abs"] / scale <= 1e-9
    sizes = np.array([c.N for c in cases])
    for i in list(np.argsort(sizes)[:2]) + list(np.argsort(sizes)[-2:]):
        o = oracle_from_case(cases[i])
        o.run(window)
        h, _ = e.get(int(i))
        assert np.max(np.abs(h - o.get_state()[0])) <= 1e-6, int(i)


def test_warm_started_step_full_size():
    case = W.heterogeneous_box(512, 512, 64, seed=2000)
    fixed = dict(dt0=300.0, f_grow=1.0)
    net = rf.Network()
    net.set_params(W.nn_init_params(7))
    sc = warmstart.scales_for(case, out_scale=1e-6)
    states = {}
    for warm in (False, True):
        s = rf.Solver.from_case(case, precision="mixed", **fixed)
        if warm:
            s.ws_attach(net, sc)
        info = s.step()
        assert info.rejected == 0
        states[warm] = s.get_state()[0]
        assert s.mass_balance()["closure_rel"] <= 1e-9
        if warm:
            assert s.ws_stats() == {"guesses": 1, "fallbacks": 0}
        s.close()
    assert np.max(np.abs(states[True] - states[False])) <= 1e-6
