"""Pins of the oracle's closures (Eq. 2-4, Eq. A6) against facts that do not
come from retyping those formulas: closed forms at special points, the
identity C = d(theta)/dh, Mualem's integral definition of the relative
conductivity, limits and monotonicity; and, at 80 heads from -1e-5 to
-1e3 m, K against Mualem's integral and C against the derivative of Eq. 2,
both in 30-digit arithmetic, to the rounding of the FP64 literal forms."""
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


# ---------------------------------------------------------------- high precision
# Independent high-precision references (mpmath, 30 digits): Mualem's integral
# for K (not Eq. 4's closed form) and the derivative of Eq. 2's retention
# curve for C (not Eq. 3).  The oracle evaluates Eq. 3 and Eq. 4 literally in
# FP64, so the tolerance follows the rounding of that literal form.
try:
    import mpmath as mp
except ImportError:                      # the other pins of this file need no mpmath
    mp = None
needs_mpmath = pytest.mark.skipif(mp is None, reason="mpmath is not installed")
EPS = np.finfo(float).eps
H_DENSE = -np.logspace(-5, 3, 80)


def _mualem_kr(s, h):
    """Mualem's K_r = Se^(1/2) [I(Se) / I(1)]^2 with I(Se) = int_0^Se dx / |h(x)|
    and |h(x)| = (x^(-1/m) - 1)^(1/n) / alpha, by tanh-sinh quadrature.  Near
    x = 1 the integrand behaves as (m / (1 - x))^(1/n); with 1 - x = t^(1/m)
    it becomes smooth in t, so the wet part is integrated in t and the wet
    end taken as I(1) minus the part over x in [Se, 1]."""
    with mp.workdps(30):
        n = mp.mpf(s["n"])
        m = 1 - 1 / n
        f = lambda x: (x ** (-1 / m) - 1) ** (-1 / n)          # alpha cancels in the ratio

        def wet(y_top):                                        # int over x in [1 - y_top, 1]
            q = 1 / m
            g = lambda t: mp.expm1(-mp.log1p(-t ** q) / m) ** (-1 / n) * q * t ** (q - 1)
            return mp.quad(g, [0, y_top ** m])

        se = (1 + (-mp.mpf(s["alpha"]) * mp.mpf(h)) ** n) ** (-m)
        half = mp.mpf(1) / 2
        i1 = mp.quad(f, [0, half]) + wet(half)
        i_se = mp.quad(f, [0, se]) if se < half else i1 - wet(1 - se)
        kr = mp.sqrt(se) * (i_se / i1) ** 2
        # pieces of the literal form, for its rounding bound
        s1 = se ** (1 / m)
        u = 1 - s1
        v = u ** m
        w = 1 - v
        return kr, float(s1), float(u), float(v), float(w), float(m)


def _literal_rounding_bound(s1, u, v, w, m):
    """Relative rounding error of Ks Se^(1/2) [1 - (1 - Se^(1/m))^m]^2 taken
    literally: Se^(1/m) carries ~5 ulp, 1 - Se^(1/m) loses s1/u of it, the
    m-th power keeps m times that, and 1 - (.)^m loses v/w; the square
    doubles it.  A factor 4 of margin."""
    rel_u = 5 * EPS * s1 / u + EPS
    rel_v = m * rel_u + EPS
    rel_w = (v / w) * rel_v + EPS
    return 4 * (2 * rel_w + 4 * EPS)


@needs_mpmath
@pytest.mark.parametrize("s", SOILS)
def test_conductivity_matches_mualem_integral_to_rounding(s):
    worst = 0.0
    for h in H_DENSE:
        kr, s1, u, v, w, m = _mualem_kr(s, h)
        K = O.closure(s, float(h))[1]
        err = abs(K / s["Ks"] / float(kr) - 1)
        bound = _literal_rounding_bound(s1, u, v, w, m)
        assert err <= bound, (h, err, bound)
        worst = max(worst, err)
    assert worst < 1e-6                       # over 1e-5 .. 1e3 m of suction


@needs_mpmath
@pytest.mark.parametrize("s", SOILS)
def test_capacity_is_the_high_precision_derivative_of_eq2(s):
    with mp.workdps(30):
        n, a = mp.mpf(s["n"]), mp.mpf(s["alpha"])
        m = 1 - 1 / n
        d = mp.mpf(s["theta_s"]) - mp.mpf(s["theta_r"])
        theta = lambda h: mp.mpf(s["theta_r"]) + d * (1 + (-a * h) ** n) ** (-m)     # Eq. 2
        for h in H_DENSE[::3]:
            ref = mp.diff(theta, mp.mpf(h))
            C = O.closure(s, float(h))[2]
            assert abs(C / float(ref) - 1) <= 1e-12, h
