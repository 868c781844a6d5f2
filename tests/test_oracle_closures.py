"""Pins of the oracle's closures (Eq. 2-4, Eq. A6) against facts that do not
come from retyping those formulas: closed forms at special points, the
identity C = d(theta)/dh, Mualem's integral definition of the relative
conductivity, limits and monotonicity."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O

LOAM = dict(model=O.VG, theta_r=0.078, theta_s=0.43, alpha=3.6, n=1.56, Ks=2.89e-6, S=1e-5)
SOILS = [
    LOAM,
    dict(model=O.VG, theta_r=0.05, theta_s=0.40, alpha=2.0, n=1.8, Ks=1e-5, S=1e-5),
    dict(model=O.VG, theta_r=0.08, theta_s=0.45, alpha=2.3, n=1.2, Ks=1e-3, S=1e-5),   # Eq. 5 layer 1
    dict(model=O.VG, theta_r=0.20, theta_s=0.50, alpha=2.1, n=2.4, Ks=1e-5, S=1e-4),   # Eq. 5 layer 2
]


@pytest.mark.parametrize("s", SOILS)
def test_saturated_branch_and_tie(s):
    # Eq. 2-4: theta = theta_s, C = S, K = Ks for h >= 0 (tie h = 0 saturated);
    # theta* continues as theta_s + S h above zero.
    th, K, C = O.closure(s, 0.0)
    assert th == s["theta_s"] and K == s["Ks"] and C == s["S"]
    th, K, C = O.closure(s, 2.5)
    assert th == pytest.approx(s["theta_s"] + s["S"] * 2.5, rel=1e-15)
    assert K == s["Ks"] and C == s["S"]


@pytest.mark.parametrize("s", SOILS)
def test_closed_form_at_unit_suction(s):
    # At -alpha h = 1: (1 + 1)^-m = 2^-m and x/(1+x) = 1/2, so
    # theta = theta_r + (theta_s - theta_r) 2^-m and
    # K = Ks 2^(-m/2) (1 - 2^-m)^2, C = (theta_s-theta_r) alpha n m 2^-(m+1).
    m = 1 - 1 / s["n"]
    h = -1.0 / s["alpha"]
    th, K, C = O.closure(s, h)
    assert th == pytest.approx(s["theta_r"] + (s["theta_s"] - s["theta_r"]) * 2 ** -m, rel=1e-14)
    assert K == pytest.approx(s["Ks"] * 2 ** (-m / 2) * (1 - 2 ** -m) ** 2, rel=1e-12)
    assert C == pytest.approx((s["theta_s"] - s["theta_r"]) * s["alpha"] * s["n"] * m * 2 ** -(m + 1), rel=1e-13)


@pytest.mark.parametrize("s", SOILS)
@pytest.mark.parametrize("h", [-1e-3, -0.05, -0.3, -1.0, -4.0, -25.0])
def test_capacity_is_derivative_of_theta(s, h):
    # C(h) must be d(theta)/dh (Eq. 3 vs Eq. 2): centred differences at two
    # step sizes combined by Richardson extrapolation (error O(eps^4)).
    def cd(eps):
        return (O.closure(s, h + eps)[0] - O.closure(s, h - eps)[0]) / (2 * eps)

    eps = 2e-3 * abs(h)
    fd = (4 * cd(eps / 2) - cd(eps)) / 3
    assert O.closure(s, h)[2] == pytest.approx(fd, rel=1e-6)


@pytest.mark.parametrize("s", SOILS[:3])
@pytest.mark.parametrize("h", [-0.02, -0.2, -0.7, -2.0, -10.0])
def test_conductivity_matches_mualem_integral(s, h):
    # Mualem's model: K_r(Se) = Se^(1/2) [ I(Se) / I(1) ]^2 with
    # I(Se) = int_0^Se dS / |h(S)|, and van Genuchten's inverse retention
    # |h(S)| = (S^(-1/m) - 1)^(1/n) / alpha, integrated by adaptive
    # quadrature.  This pins Eq. 4, including its garbled exponent.
    n, a = s["n"], s["alpha"]
    m = 1 - 1 / n
    se = (1 + (-a * h) ** n) ** (-m)

    def integrand(S):
        return a / (S ** (-1 / m) - 1) ** (1 / n)

    def I(upper):
        v, _ = integrate.quad(integrand, 0.0, upper, limit=400, epsabs=0, epsrel=1e-12)
        return v

    # I(1) has an integrable singularity at S = 1
    i1, _ = integrate.quad(integrand, 0.0, 1.0, limit=800, epsabs=0, epsrel=1e-11)
    kr = math.sqrt(se) * (I(se) / i1) ** 2
    K = O.closure(s, h)[1]
    assert K / s["Ks"] == pytest.approx(kr, rel=2e-7)


@pytest.mark.parametrize("s", SOILS)
def test_limits_and_monotonicity(s):
    hs = -np.logspace(-4, 3, 200)[::-1]          # from -1000 m up to -1e-4 m
    vals = np.array([O.closure(s, h) for h in hs])
    th, K = vals[:, 0], vals[:, 1]
    assert np.all(np.diff(th) > 0) and np.all(np.diff(K) > 0)
    # far dry end: Se -> (-alpha h)^-(n-1), i.e. theta -> theta_r
    se0 = (th[0] - s["theta_r"]) / (s["theta_s"] - s["theta_r"])
    assert se0 * (s["alpha"] * 1e3) ** (s["n"] - 1) == pytest.approx(1.0, rel=1e-3)
    # wet end: (-alpha h)^n -> 0 gives K/Ks -> (1 - (-alpha h)^(n-1))^2
    assert K[-1] / s["Ks"] == pytest.approx((1 - (s["alpha"] * 1e-4) ** (s["n"] - 1)) ** 2, rel=1e-3)
    assert th[-1] == pytest.approx(s["theta_s"], rel=1e-3)
    assert np.all(vals[:, 2] > 0)


def test_gardner_closed_forms():
    # Eq. A6: K = Ks exp(alpha h); the retention curve read for this model is
    # theta_r + (theta_s - theta_r) exp(alpha h), so C = (theta_s-theta_r) alpha exp(alpha h).
    g = dict(model=O.GARDNER, theta_r=0.05, theta_s=0.4, alpha=0.06, Ks=1e-6, S=1e-5)
    for h in (-0.1, -1.0, -7.5):
        th, K, C = O.closure(g, h)
        assert K == pytest.approx(1e-6 * math.exp(0.06 * h), rel=1e-15)
        assert th == pytest.approx(0.05 + 0.35 * math.exp(0.06 * h), rel=1e-15)
        eps = 1e-6
        fd = (O.closure(g, h + eps)[0] - O.closure(g, h - eps)[0]) / (2 * eps)
        assert C == pytest.approx(fd, rel=1e-7)
    assert O.closure(g, 0.0) == (0.4, 1e-6, 1e-5)
