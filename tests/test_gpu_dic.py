"""The red-black DIC preconditioner of the FP32 inner PCG (Sec. 2.2's
preconditioner, cells eliminated by colour) against the oracle: the mixed
path with DIC reaches the oracle's states (<= 1e-6 m) with the same step and
Picard sequences as Jacobi; on a stiff saturated block it solves the system
to the oracle's dense solution in fewer inner iterations than Jacobi; FP64
with DIC is refused."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1809_10895_gb300 import rf
from paper_1809_10895_gb300 import workloads as W
from tests.helpers import oracle_from_case
from tests.test_gpu_parity import TOL_MIXED, gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1809_10895_gb300 import build as B
    B.build()
    rf.load()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("mk,t_end", [
    (lambda: W.heterogeneous_box(21, 13, 17, d=0.25, seed=7, water_table_depth=2.0, rain=4e-6, rain_hours=1.0),
     4 * 3600.0),
    (lambda: W.watershed(24, 20, 16, dx=10.0, dz=0.5, seed=3, hours=24), 12 * 3600.0)])
def test_mixed_dic_run_matches_oracle(mk, t_end):
    case = mk()
    runs = {}
    for pc in ("jacobi", "dic"):
        s = rf.Solver.from_case(case, precision="mixed", precond=pc)
        steps = s.run(t_end)
        runs[pc] = (s.get_state()[0], [(st.dt, st.picard, st.rejected) for st in steps], s.mass_balance())
    o = oracle_from_case(case)
    o.run(t_end)
    ho = o.get_state()[0]
    act = np.asarray(case.active, bool) if case.active is not None else slice(None)
    assert runs["dic"][1] == runs["jacobi"][1]
    assert np.max(np.abs(runs["dic"][0] - ho)[act]) <= TOL_MIXED
    assert runs["dic"][2]["closure_rel"] <= 1e-9


def test_dic_cuts_inner_iterations_on_a_stiff_block():
    case = W.heterogeneous_box(16, 12, 10, seed=5)
    case.h0 = np.full(case.N, 0.5)                      # saturated: tiny storage
    case.soils = [dict(sl, S=1e-6) for sl in case.soils]
    o = oracle_from_case(case, tol_cg=1e-10, cg_max_it=20000)
    xd, _, _ = o.solve(case.h0, case.h0, 3600.0, dense=True)
    its = {}
    for pc in ("jacobi", "dic"):
        s = rf.Solver.from_case(case, precision="mixed", precond=pc, tol_cg=1e-10, cg_max_it=20000)
        s.assemble(gpu(case.h0), gpu(case.h0), 3600.0, 0.0)
        x = gpu(case.h0)
        its[pc] = s.solve(x)
        assert np.max(np.abs(x.cpu().numpy()[o.active_cells] - xd)) <= 1e-8 * np.max(np.abs(xd))
    assert its["dic"] <= 0.75 * its["jacobi"]


def test_fp64_with_dic_is_refused():
    case = W.heterogeneous_box(8, 8, 4, seed=1)
    with pytest.raises(RuntimeError):
        rf.Solver.from_case(case, precision="fp64", precond="dic")
