"""The seeded input recipes have the properties their builders document:
deterministic per seed, the stated sizes and ranges, and field statistics
(the Gaussian random field's variance and correlation length, the terrain's
range, the storm series' structure)."""
import numpy as np
import pytest

from paper_1809_10895_gb300 import workloads as W


def _fingerprint(c):
    parts = [c.h0]
    for x in (c.Ks_cell, c.active, c.zone_of_cell):
        if x is not None:
            parts.append(np.asarray(x, np.float64))
    parts.append(np.array([v for s in c.soils for v in (s["alpha"], s.get("n", 0.0), s["Ks"])]))
    for bc in c.bcs:
        if bc.v is not None:
            parts += [np.asarray(bc.t, np.float64), np.asarray(bc.v, np.float64)]
    return np.concatenate([np.ravel(p) for p in parts])


def test_recipes_are_deterministic_per_seed():
    for mk in (lambda s: W.heterogeneous_box(16, 12, 8, seed=s), lambda s: W.watershed(32, 16, 40, seed=s, hours=48),
               lambda s: W.ensemble(4, seed=s)[3]):
        a, b, c = _fingerprint(mk(3)), _fingerprint(mk(3)), _fingerprint(mk(4))
        np.testing.assert_array_equal(a, b)
        assert a.shape != c.shape or not np.array_equal(a, c)


def test_random_field_statistics():
    # unit variance and an exponential covariance of correlation length 8 cells
    g = W.gaussian_random_field((64, 64, 32), 8.0, seed=5).reshape(32, 64, 64)
    assert abs(g.mean()) < 0.25 and g.var() == pytest.approx(1.0, rel=1e-6)
    for lag in (4, 8):
        rho = np.mean(g[:, :, :-lag] * g[:, :, lag:]) / g.var()
        assert rho == pytest.approx(np.exp(-lag / 8.0), abs=0.15)


def test_box_recipe():
    c = W.heterogeneous_box(32, 32, 16, seed=2)
    lnK = np.log(c.Ks_cell)
    assert lnK.std() == pytest.approx(1.0, rel=0.05)          # sigma_lnK = 1 (unit-variance field)
    assert lnK.mean() == pytest.approx(np.log(1e-5), abs=0.5)
    z = c.z_centres()
    np.testing.assert_allclose(c.h0 + z, c.h0[0] + z[0])       # hydrostatic start
    assert c.N == 32 * 32 * 16 and c.dx == c.dy == c.dz == 0.25


def test_watershed_recipe():
    c = W.watershed(64, 48, 64, seed=1, hours=720)
    act = c.active.reshape(c.nz, c.ny, c.nx).astype(bool)
    top = act.sum(axis=0) * c.dz                               # active depth per column
    assert top.min() >= 16.0 - c.dz and top.max() <= 32.0 + c.dz
    assert len(c.soils) == 4
    for s in c.soils:
        assert 0.5 <= s["alpha"] <= 5.0 and 1.2 <= s["n"] <= 2.5 and 1e-7 <= s["Ks"] <= 1e-4
    rain = next(b for b in c.bcs if b.face == "zmax")
    assert np.all(rain.v >= 0.0) and np.any(rain.v > 0.0) and np.any(rain.v == 0.0)


def test_ensemble_recipe():
    cases = W.ensemble(64, seed=0)
    for c in cases:
        assert 1 <= c.nx <= 16 and 1 <= c.ny <= 16 and 50 <= c.nz <= 400 and c.dz == 0.01
        s = c.soils[0]
        assert 0.5 <= s["alpha"] <= 5.0 and 1.2 <= s["n"] <= 2.5 and 1e-7 <= s["Ks"] <= 1e-4
        assert -3.0 <= c.h0[0] <= -0.1 and np.all(c.h0 == c.h0[0])
    assert len({(c.nx, c.ny, c.nz) for c in cases}) > 32       # uneven sizes


def test_column_and_slope_recipes():
    col = W.infiltration_column()
    assert (col.nx, col.ny, col.nz, col.dz) == (1, 1, 200, 0.005) and np.all(col.h0 == -1.0)
    sl = W.tilted_slope(nx=8, ny=8, nz=50)
    assert np.linalg.norm(sl.gravity) == pytest.approx(1.0) and sl.nz * sl.dz == pytest.approx(10.0)
    assert np.degrees(np.arcsin(sl.gravity[0])) == pytest.approx(20.0)
    assert np.all(sl.h0 == -10.0)
