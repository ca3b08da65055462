"""Pins of the oracle's heterogeneous backgrounds B1/B2 (Sec. 5; CPU only).

The collision rate is written out here a second time from the paper's
definition of B1 and B2, and the flight inversion of eq. intinv is checked
against numerical quadrature of that definition and against a brute-force
simulation of the collision process.  With a = 0 the background is
homogeneous (R = b, mu = 0, sigma = 1) and the oracle's heterogeneous path
must give the homogeneous path.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle as O


def R_paper(kind, a, b, x):
    """R_1 / R_2 of Sec. 5, as printed."""
    if kind == O.BG_B1:
        return -b * (a * (x - 1.0) - 1.0) if x <= 1.0 else b * (a * (x - 1.0) + 1.0)
    return b if x <= 1.0 else b * (a * (x - 1.0) + 1.0)


CASES = [(O.BG_B1, 10.0, 100.0), (O.BG_B1, 0.5, 3.0), (O.BG_B2, 20.0, 10.0), (O.BG_B2, 2.0, 1000.0)]


@pytest.mark.parametrize("kind,a,b", CASES)
def test_rate_matches_the_papers_definition(kind, a, b):
    bg = O.het_bg(kind, a, b)
    for x in np.linspace(-3.0, 4.0, 71):
        assert O.het_R(bg, float(x)) == pytest.approx(R_paper(kind, a, b, float(x)), rel=1e-15)


@pytest.mark.parametrize("kind,a,b", CASES)
def test_flight_inversion_against_quadrature(kind, a, b):
    """eq. intinv: int_0^tau R(x0 + v t) dt = E, by adaptive quadrature of the
    printed rate, for starts on both sides of the kink at x = 1, both
    directions, flights that cross the kink and flights that do not."""
    bg = O.het_bg(kind, a, b)
    rng = np.random.default_rng(1)
    dt = 0.01
    for _ in range(200):
        x0 = float(rng.uniform(0.0, 2.0))
        v = float(rng.normal()) * 3.0
        E = float(rng.exponential())
        u = O.het_flight(bg, x0, v, dt, E)
        tau = u * dt
        kink = (1.0 - x0) / v if v != 0 else -1.0
        pts = [kink] if 0.0 < kink < tau else None
        got, _ = integrate.quad(lambda t: R_paper(kind, a, b, x0 + v * t), 0.0, tau, points=pts,
                                epsabs=0, epsrel=1e-13, limit=200)
        assert got == pytest.approx(E, rel=1e-10, abs=1e-13), (x0, v, E, tau)
        # the depth function is the same integral, also behind the start
        for w in (0.3 * u, -0.7 * u):
            lo, hi = sorted((0.0, w * dt))
            k = [kink] if lo < kink < hi else None
            q, _ = integrate.quad(lambda t: R_paper(kind, a, b, x0 + v * t), lo, hi, points=k,
                                  epsabs=0, epsrel=1e-13, limit=200)
            assert O.het_depth(bg, x0, v, dt, w) == pytest.approx(math.copysign(q, w), rel=1e-10,
                                                                  abs=1e-13)


@pytest.mark.parametrize("x0,v", [(0.7, 2.0), (1.3, -1.5), (1.0, 0.8), (0.2, -1.0)])
def test_flight_law_against_brute_force_collisions(x0, v):
    """Collision times of the process with rate R(x0 + v t), simulated by
    thinning a Poisson process of a dominating constant rate, have the law of
    the inverted flights tau(E), E ~ Exp(1)."""
    kind, a, b = O.BG_B1, 4.0, 2.0
    bg = O.het_bg(kind, a, b)
    rng = np.random.default_rng(7)
    n = 20000
    dt = 0.01
    inv = np.array([O.het_flight(bg, x0, v, dt, float(E)) * dt for E in rng.exponential(size=n)])
    tmax = float(np.max(inv)) * 1.5
    rmax = max(R_paper(kind, a, b, x0), R_paper(kind, a, b, x0 + v * tmax), b)
    brute = np.empty(n)
    for i in range(n):
        t = 0.0
        while True:
            t += rng.exponential(1.0 / rmax)
            if rng.random() * rmax <= R_paper(kind, a, b, x0 + v * t):
                break
        brute[i] = t
    assert stats.ks_2samp(inv, brute).pvalue > 1e-3


def test_a_zero_reduces_to_the_homogeneous_path(orc):
    """a = 0: R = b everywhere, the homogeneous background with mu = 0,
    sigma = 1.  Single paths are the homogeneous oracle's bit for bit; pairs
    have the same event counts and positions to 1e-12 (the coarse flight of
    eq. epsilon-update is formed as E - R dt (t_c - t_kappa) then divided by
    R dt, not as the difference of flights, so it rounds differently)."""
    b, T, dt0, M = 7.0, 1.0, 0.25, 2
    for kind in (O.BG_B1, O.BG_B2):
        for level in (0, 1, 3):
            het = O.het_pairs(kind, 0.0, b, T, dt0, M, level, level > 0, 5, 3000, x0=0.0,
                              threads=8)
            d = O.LevelDesc()
            d.R, d.mu, d.sigma = b, 0.0, 1.0
            d.dt, d.n, d.M, d.level = dt0 / M ** level, int(T / dt0) * M ** level, M, level
            d.init, d.recipe, d.seed, d.request, d.coupled = 0, O.RECIPE_53, 0, 0, 1 if level else 0
            xf = np.zeros(3000); xc = np.zeros(3000)
            ef = np.zeros(3000, np.int64); ec = np.zeros(3000, np.int64)
            import ctypes
            P = lambda a_, t: a_.ctypes.data_as(ctypes.POINTER(t))
            assert orc.lib().orc_pairs(ctypes.byref(d), 5, 3000, P(xf, ctypes.c_double),
                                       P(xc, ctypes.c_double), P(ef, ctypes.c_int64),
                                       P(ec, ctypes.c_int64)) == 0
            assert np.array_equal(het[2], ef) and np.array_equal(het[3], ec)
            if level == 0:
                assert np.array_equal(het[0], xf)
            else:
                assert np.all(np.abs(het[0] - xf) <= 1e-12 * np.maximum(1, np.abs(xf)))
                assert np.all(np.abs(het[1] - xc) <= 1e-12 * np.maximum(1, np.abs(xc)))


@pytest.mark.parametrize("a,b", [(10.0, 100.0), (1.0, 10.0)])
def test_symmetric_background_gives_mean_position_one(a, b):
    """B1 is symmetric about x = 1 and so is the velocity law: the KD path
    from x0 = 1 has E[x(T)] = 1 on every level, fine and coarse, and the
    level difference E[x_l - x_{l-1}] = 0 (the paper's QoI is x(T))."""
    n = 40000
    for level in (0, 2, 4):
        xf, xc, _, _ = O.het_pairs(O.BG_B1, a, b, 1.0, 0.5, 2, level, level > 0, 0, n, threads=8)
        se = xf.std() / math.sqrt(n)
        assert abs(xf.mean() - 1.0) < 4.5 * se
        if level:
            assert abs(xc.mean() - 1.0) < 4.5 * xc.std() / math.sqrt(n)
            y = xf - xc
            assert abs(y.mean()) < 4.5 * y.std() / math.sqrt(n) + 1e-15


def test_asymmetric_background_drifts_into_the_low_rate_side():
    """B2 has the constant rate b left of x = 1 and a growing rate right of
    it; with a > 0 particles spread further to the left, so E[x(T)] < 1, and
    the fine and coarse paths agree on it (telescoping)."""
    n = 40000
    xf, xc, _, _ = O.het_pairs(O.BG_B2, 20.0, 10.0, 1.0, 0.5, 2, 3, True, 0, n, threads=8)
    assert xf.mean() < 1.0 - 6 * xf.std() / math.sqrt(n)
    assert abs(xf.mean() - xc.mean()) < 4.5 * (xf - xc).std() / math.sqrt(n) + 0.01


@pytest.mark.parametrize("kind,a,b,level", [(O.BG_B1, 10.0, 30.0, 2), (O.BG_B1, 10.0, 1000.0, 4)])
def test_coarse_path_has_the_single_level_law(kind, a, b, level):
    """In the symmetric background B1 the coarse path of a correlated pair is
    distributed as an independent single-level path at the coarse step (the
    telescoping of eq. telsum; the coarse random numbers keep their laws,
    Sec. 5.1).  Two-sample KS and Anderson-Darling on x(T), n = 20000
    each."""
    n = 20000
    _, xc, _, _ = O.het_pairs(kind, a, b, 1.0, 0.5, 2, level, True, 0, n, threads=8)
    xs, _, _, _ = O.het_pairs(kind, a, b, 1.0, 0.5, 2, level - 1, False, 0, n, seed=99, threads=8)
    assert stats.ks_2samp(xc, xs).pvalue > 1e-3
    assert stats.anderson_ksamp([xc, xs]).pvalue > 1e-3


def test_coarse_draws_of_table_hypothesis_background():
    """Sec. 5.1 on the oracle for the background of Table hypothesis (B1,
    a = 10, b = 1000): nu~ ~ N(0,1), E~ ~ Exp(1), chi~ ~ N(0,1) by A^2 at
    N = 1000 (the paper's size) and at N = 50000, for l = 5 (M = 2) and
    l = 7 (M = 8)."""
    from ad_test import ad_pvalue, ad_statistic
    for level, M in ((5, 2), (7, 8)):
        nu, E, chi = O.het_coarse_draws(O.BG_B1, 10.0, 1000.0, 1.0, 1.0, 2, level, 0, 400000, 50000,
                                        request=level, coarsening=M)
        assert len(nu) == 50000
        for N in (1000, 50000):
            assert ad_pvalue(ad_statistic(nu[:N], stats.norm.cdf)) > 1e-3
            assert ad_pvalue(ad_statistic(E[:N], stats.expon.cdf)) > 1e-3
            assert ad_pvalue(ad_statistic(chi[:N], stats.norm.cdf)) > 1e-3


def test_asymmetric_background_biases_the_coarse_velocity():
    """A property of the coupling as printed, recorded here: in the
    asymmetric background B2 the fine kinetic phase kappa that spans the end
    of a coarse step is length-biased (a longer flight is likelier to span a
    given time), and flight length depends on the velocity (a particle moving
    into the low-rate side x < 1 flies longer).  So nu~ = nu_kappa of eq.
    nu-update leans negative, and the coarse path of a pair drifts left of an
    independent single-level path at the same step.  With a = 0 both effects
    vanish (flight length no longer depends on the velocity)."""
    nu, E, chi = O.het_coarse_draws(O.BG_B2, 20.0, 10.0, 1.0, 0.5, 2, 3, 0, 200000, 50000)
    se = nu.std() / math.sqrt(len(nu))
    assert nu.mean() < -5 * se
    nu0, _, _ = O.het_coarse_draws(O.BG_B2, 0.0, 10.0, 1.0, 0.5, 2, 3, 0, 200000, 50000)
    assert abs(nu0.mean()) < 4.5 * nu0.std() / math.sqrt(len(nu0))
