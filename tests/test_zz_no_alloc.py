"""rf_pcg_solve_noalloc: the linear solve for callers that cannot allocate
device memory (applications that own the device memory pool and forbid
cudaMalloc inside their time loop, or that must avoid its implicit device
synchronisation).  It keeps its work vectors in a fixed file-scope device
array instead of allocating.

Checked through the C ABI against the context solver's rf_solve (FP64 PCG)
on the same assembled systems, two calls in a row, with the solve tolerance
the parity tests use.  Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1809_10895_gb300 import rf
from paper_1809_10895_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1809_10895_gb300 import build as B
    B.build()
    rf.load()
    torch.cuda.set_device(0)


def _faces(K, case):
    """Upper-face coefficients T = (K_P + K_N)/2 * A/d of an all-active grid."""
    nx, ny, nz = case.nx, case.ny, case.nz
    K3 = K.view(nz, ny, nx)
    Tx = torch.zeros_like(K3)
    Ty = torch.zeros_like(K3)
    Tz = torch.zeros_like(K3)
    Tx[:, :, :-1] = 0.5 * (K3[:, :, :-1] + K3[:, :, 1:]) * (case.dy * case.dz / case.dx)
    Ty[:, :-1, :] = 0.5 * (K3[:, :-1, :] + K3[:, 1:, :]) * (case.dx * case.dz / case.dy)
    Tz[:-1, :, :] = 0.5 * (K3[:-1, :, :] + K3[1:, :, :]) * (case.dx * case.dy / case.dz)
    return Tx.reshape(-1).contiguous(), Ty.reshape(-1).contiguous(), Tz.reshape(-1).contiguous()


def test_noalloc_solve_matches_context_solve_twice():
    case = W.heterogeneous_box(21, 13, 17, d=0.25, seed=11, water_table_depth=2.0, rain=4e-6, tol_cg=1e-13)
    s = rf.Solver.from_case(case)
    rng = np.random.default_rng(4)
    dev = dict(dtype=torch.float64, device="cuda")
    for call, dt in enumerate((30.0, 240.0)):
        hk = case.h0 + rng.normal(0, 0.02, case.N)
        hk_t = torch.as_tensor(hk, **dev)
        K = torch.zeros(case.N, **dev)
        b = torch.zeros(case.N, **dev)
        diag = torch.zeros(case.N, **dev)
        s.assemble(hk_t, torch.as_tensor(case.h0, **dev), dt, 0.0, K=K, b=b, diag=diag)
        Tx, Ty, Tz = _faces(K, case)
        x_ref = hk_t.clone()
        s.solve(x_ref)                                   # existing entry point
        x = hk_t.clone()
        it = rf.pcg_solve_noalloc((case.nx, case.ny, case.nz), diag, Tx, Ty, Tz, b, x, tol=1e-13)
        assert it > 0, call
        assert torch.max(torch.abs(x - x_ref)).item() <= 1e-10, call


def test_noalloc_rejects_grids_beyond_its_array():
    dev = dict(dtype=torch.float64, device="cuda")
    n = rf.NOALLOC_MAX_CELLS + 1
    v = torch.ones(n, **dev)
    with pytest.raises(rf.RFError) as e:
        rf.pcg_solve_noalloc((n, 1, 1), v, v, v, v, v, v.clone())
    assert e.value.status == rf.RF_ERR_ARG
