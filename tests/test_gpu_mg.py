"""Multigrid-preconditioned FP32 inner PCG (mixed path): same solutions as the
Jacobi-preconditioned solve and the CPU oracle, far fewer inner iterations on
a stiff anisotropic system, and step-level parity on a masked watershed."""
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


def stiff_case():
    # saturated, heterogeneous, 10:1 anisotropic cells, storage-poor: the
    # capacity term is far below the face conductances (ill-conditioned)
    nx, ny, nz = 37, 29, 33
    rng = np.random.default_rng(12)
    Ks = np.exp(np.log(1e-4) + 1.5 * rng.standard_normal(nx * ny * nz))
    c = W.Case(name="stiff", nx=nx, ny=ny, nz=nz, dx=1.0, dy=1.0, dz=0.1,
               soils=[dict(model="vg", theta_r=0.05, theta_s=0.4, alpha=2.0, n=1.8, Ks=1e-4, S=1e-6)],
               Ks_cell=Ks, params=W.default_params(tol_cg=1e-10))
    c.h0 = (nz * 0.1 + 2.0) - c.z_centres()
    c.bcs = [W.BC("zmin", "dirichlet", np.array([0.0]), np.array([nz * 0.1 + 1.5])),
             W.BC("zmax", "flux", np.array([0.0]), np.array([5e-5]))]
    return c


@pytest.mark.parametrize("dt", [60.0, 3600.0])
def test_mg_solve_matches_and_beats_jacobi(dt):
    case = stiff_case()
    dev = dict(dtype=torch.float64, device="cuda")
    hk = torch.as_tensor(case.h0, **dev)
    x0 = torch.zeros(case.N, **dev)
    sols, its = {}, {}
    for pc in ("jacobi", "mg"):
        s = rf.Solver.from_case(case, precision="mixed", precond=pc)
        s.assemble(hk, hk, dt, 0.0)
        x = x0.clone()
        its[pc] = s.solve(x)
        sols[pc] = x.cpu().numpy()
    o = oracle_from_case(case, tol_cg=1e-13)
    xo, ito, _ = o.solve(case.h0, case.h0, dt, x0=np.zeros(case.N))
    scale = np.abs(xo).max()
    for pc in ("jacobi", "mg"):
        assert np.max(np.abs(sols[pc] - xo)) <= 1e-8 * scale, pc
    assert its["mg"] * 4 <= its["jacobi"], its


def test_mg_watershed_parity():
    case = W.watershed(24, 20, 16, dx=10.0, dz=0.5, seed=0, hours=60, tol_cg=1e-12)
    s = rf.Solver.from_case(case, precision="mixed", precond="mg")
    o = oracle_from_case(case)
    t_end = 24 * 3600.0          # through the first storm of this seed (hours 11-20)
    sg = s.run(t_end)
    so = o.run(t_end)
    assert len(sg) == len(so)
    assert [a.picard for a in sg] == [b.picard for b in so]
    hg, _ = s.get_state()
    ho, _ = o.get_state()
    act = case.active.astype(bool)
    assert np.max(np.abs(hg - ho)[act]) <= 1e-6
