"""The oracle's OpenMP build (the same C source with -fopenmp, used for the
all-core CPU baseline) against its one-thread build: the per-cell loops are
independent and only sums over cells change their order, so both builds take
the same steps with the same Picard counts and agree to rounding."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1809_10895_gb300 import workloads as W
from tests.helpers import oracle_from_case

THREADS = O.num_threads(openmp=True)
pytestmark = pytest.mark.skipif(THREADS < 1, reason="gcc cannot build the oracle with -fopenmp here")


def test_thread_counts():
    assert O.num_threads(openmp=False) == 1
    assert THREADS >= 1
    if (os.cpu_count() or 1) > 1 and "OMP_NUM_THREADS" not in os.environ:
        assert THREADS > 1


@pytest.mark.parametrize("mk,n_steps", [
    (lambda: W.heterogeneous_box(21, 13, 17, d=0.25, seed=7, water_table_depth=2.0, rain=4e-6), 12),
    (lambda: W.watershed(24, 20, 16, dx=10.0, dz=0.5, seed=3, hours=24), 8),
    (lambda: W.infiltration_column(nz=60, dz=0.01), 20),
])
def test_openmp_build_takes_the_same_steps(mk, n_steps):
    case = mk()
    one, many = oracle_from_case(case), oracle_from_case(case, openmp=True)
    for _ in range(n_steps):
        a, b = one.step(), many.step()
        assert (a.dt, a.t, a.picard, a.rejected) == (b.dt, b.t, b.picard, b.rejected)
        assert abs(a.cg - b.cg) <= a.picard          # a CG stop may move by one iteration per solve
    h1, m1 = one.get_state()
    h2, m2 = many.get_state()
    act = case.active.ravel() != 0 if case.active is not None else slice(None)
    assert np.max(np.abs(h1[act] - h2[act])) <= 1e-9
    b1, b2 = one.mass_balance(), many.mass_balance()
    for k in b1:
        assert b2[k] == pytest.approx(b1[k], rel=1e-9, abs=1e-12), k
