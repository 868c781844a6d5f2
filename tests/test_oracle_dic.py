"""Pins of the oracle's DIC-preconditioned CG (Sec. 2.2: PCG with the
diagonal incomplete Cholesky preconditioner), in the paper's natural cell
order and in the red-black order a parallel version eliminates in.

A tridiagonal matrix (one column of cells, natural order) has no fill-in,
so its incomplete factorisation is the exact one and PCG converges in one
iteration; every ordering solves the same system as the dense Cholesky
factorisation to the CG tolerance; on a stiff saturated block DIC cuts the
iterations of Jacobi-PCG (the reason the paper uses it); a whole run with
DIC takes the same steps and Picard iterations as with Jacobi."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1809_10895_gb300 import workloads as W
from tests.helpers import oracle_from_case

METHODS = (O.SOLVER_PCG, O.SOLVER_DIC, O.SOLVER_DIC_RB)


def _perturbed(case, seed=1, sd=0.02):
    return case.h0 + np.random.default_rng(seed).normal(0, sd, case.N)


def test_column_natural_dic_is_exact():
    case = W.infiltration_column(nz=60, dz=0.01)
    o = oracle_from_case(case, tol_cg=1e-12)
    hk = _perturbed(case)
    xd, _, _ = o.solve(hk, case.h0, 60.0, dense=True)
    x, it, _ = o.solve(hk, case.h0, 60.0, method=O.SOLVER_DIC)
    assert it == 1
    np.testing.assert_allclose(x, xd, rtol=0, atol=1e-12 * np.max(np.abs(xd)))
    # red-black order fills in, so it is not exact on the same matrix
    _, it_rb, _ = o.solve(hk, case.h0, 60.0, method=O.SOLVER_DIC_RB)
    assert it_rb > 1


@pytest.mark.parametrize("mk", [lambda: W.heterogeneous_box(12, 10, 8, seed=3),
                                lambda: W.watershed(12, 10, 12, dx=10.0, dz=0.5, seed=3, hours=24)])
def test_every_ordering_solves_the_system(mk):
    case = mk()
    o = oracle_from_case(case, tol_cg=1e-12)
    hk = _perturbed(case)
    xd, _, _ = o.solve(hk, case.h0, 60.0, dense=True)
    its = {}
    for m in METHODS:
        x, its[m], _ = o.solve(hk, case.h0, 60.0, method=m)
        assert its[m] >= 1
        np.testing.assert_allclose(x, xd, rtol=0, atol=1e-10 * np.max(np.abs(xd)))
    assert its[O.SOLVER_DIC] <= its[O.SOLVER_PCG] and its[O.SOLVER_DIC_RB] <= its[O.SOLVER_PCG]


def test_dic_cuts_iterations_on_a_stiff_saturated_block():
    case = W.heterogeneous_box(16, 12, 10, seed=5)
    case.h0 = np.full(case.N, 0.5)                      # saturated: tiny storage, Laplacian-like A
    case.soils = [dict(s, S=1e-6) for s in case.soils]
    o = oracle_from_case(case, tol_cg=1e-10, cg_max_it=20000)
    xd, _, _ = o.solve(case.h0, case.h0, 3600.0, dense=True)
    its = {}
    for m in METHODS:
        x, its[m], _ = o.solve(case.h0, case.h0, 3600.0, method=m)
        assert np.max(np.abs(x - xd)) <= 1e-9 * np.max(np.abs(xd))
    assert its[O.SOLVER_DIC] <= 0.5 * its[O.SOLVER_PCG]
    assert its[O.SOLVER_DIC_RB] <= 0.75 * its[O.SOLVER_PCG]


def test_run_with_dic_takes_the_same_steps():
    case = W.heterogeneous_box(12, 10, 8, seed=3)
    runs = {}
    for m in (O.SOLVER_PCG, O.SOLVER_DIC):
        o = oracle_from_case(case, solver=m)
        steps = o.run(3600.0)
        runs[m] = (o.get_state()[0], [(s.dt, s.picard, s.rejected) for s in steps], sum(s.cg for s in steps))
    assert runs[O.SOLVER_PCG][1] == runs[O.SOLVER_DIC][1]
    assert np.max(np.abs(runs[O.SOLVER_PCG][0] - runs[O.SOLVER_DIC][0])) <= 1e-8
    assert runs[O.SOLVER_DIC][2] < runs[O.SOLVER_PCG][2]
