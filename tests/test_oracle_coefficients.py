"""Pins of the oracle's homogeneous KD coefficients (CPU only).

The paper defines a and d (eqs. advection, diffusion) as the mean and the
standard deviation of the kinetic displacement over the diffusive phase,
conditioned on the velocity at its end (Sec. 2); zeta as the expected time
the final velocity acts in that phase, and beta (eq. weights-beta) as the
unconditioned standard deviation over theta' (Sec. 3.2).  The tests below
simulate that kinetic process directly (exponential collision times, fresh
Maxwellian velocities) and compare, so a dropped term, a wrong sign or a
wrong coefficient in the oracle's formulas fails one of them.  The Taylor
branches are pinned to the closed forms where both are accurate, and to a
50-digit evaluation of the closed forms at small arguments.
"""
import math

import numpy as np
import pytest


def kinetic_process(rng, R, mu, sigma, theta, n):
    """Displacement over [0, theta] of a particle that has just collided
    (fresh velocity), with later collisions at rate R; also its final velocity
    and the time the final velocity has acted."""
    v = mu + sigma * rng.standard_normal(n)
    t = np.zeros(n)
    dx = np.zeros(n)
    age = np.zeros(n)
    active = np.ones(n, bool)
    while active.any():
        idx = np.nonzero(active)[0]
        flight = rng.exponential(1.0 / R, idx.size)
        remaining = theta - t[idx]
        ends = flight >= remaining
        seg = np.where(ends, remaining, flight)
        dx[idx] += v[idx] * seg
        t[idx] += seg
        age[idx] = np.where(ends, age[idx] + seg, 0.0)
        coll = idx[~ends]
        v[coll] = mu + sigma * rng.standard_normal(coll.size)
        active[idx[ends]] = False
    return dx, v, age


@pytest.mark.parametrize("R,theta,mu,sigma", [(4.0, 0.25, 0.0, 2.0), (10.0, 0.3, 0.0, 1.0),
                                              (1.0, 0.4, 0.7, 1.5), (50.0, 0.1, -0.3, 3.0)])
def test_advection_and_diffusion_are_conditional_moments(orc, R, theta, mu, sigma):
    L = orc.lib()
    rng = np.random.default_rng(12345)
    n = 1_500_000
    dx, v_end, _ = kinetic_process(rng, R, mu, sigma, theta, n)
    w = v_end - mu
    # conditional mean is affine in the final velocity: regress
    slope = np.dot(w - w.mean(), dx - dx.mean()) / np.dot(w - w.mean(), w - w.mean())
    intercept = dx.mean() - slope * w.mean()
    a_mu = L.orc_advection(R, mu, theta, mu)
    a_slope = L.orc_advection(R, mu, theta, mu + 1.0) - a_mu
    sd_a = math.sqrt(np.var(dx) / n)
    assert abs(intercept - a_mu) < 5 * sd_a
    assert abs(slope - a_slope) < 5 * sd_a / np.std(w) + 1e-3 * abs(a_slope)
    # conditional variance is quadratic in (v_end - mu): regress r^2 on w^2
    r2 = (dx - (a_mu + a_slope * w)) ** 2
    X = np.stack([np.ones(n), w * w], 1)
    coef, *_ = np.linalg.lstsq(X, r2, rcond=None)
    d0 = L.orc_diffusion(R, mu, sigma, theta, mu) ** 2
    d1 = L.orc_diffusion(R, mu, sigma, theta, mu + 1.0) ** 2 - d0
    assert coef[0] == pytest.approx(d0, rel=0.03)
    assert coef[1] == pytest.approx(d1, rel=0.05)


@pytest.mark.parametrize("R,theta", [(4.0, 0.25), (1.0, 2.0), (100.0, 0.05)])
def test_zeta_is_expected_time_of_final_velocity(orc, R, theta):
    rng = np.random.default_rng(7)
    _, _, age = kinetic_process(rng, R, 0.0, 1.0, theta, 1_000_000)
    zeta = orc.lib().orc_zeta(R, theta)
    assert abs(age.mean() - zeta) < 5 * age.std() / math.sqrt(age.size)


@pytest.mark.parametrize("R,theta,sigma", [(4.0, 0.25, 2.0), (10.0, 0.5, 1.0), (1.0, 0.2, 1.0)])
def test_beta_is_unconditioned_std(orc, R, theta, sigma):
    """beta_m = std of the kinetic displacement over theta'_m (mu = 0)."""
    L = orc.lib()
    tp = L.orc_theta_prime(R, theta)
    rng = np.random.default_rng(99)
    dx, _, _ = kinetic_process(rng, R, 0.0, sigma, tp, 1_000_000)
    beta = L.orc_beta(R, sigma, tp)
    assert np.std(dx) == pytest.approx(beta, rel=0.01)


def test_theta_prime_is_theta_minus_zeta(orc):
    L = orc.lib()
    for R, th in [(4.0, 0.25), (1.0, 3.0), (1e4, 1e-3), (2.0, 0.9)]:
        assert L.orc_theta_prime(R, th) == pytest.approx(th - L.orc_zeta(R, th), rel=1e-12, abs=1e-15)


def _closed(name, s):
    e = math.exp(-s)
    if name == "f":
        return 2 * (e - 1) + s * (e + 1)
    if name == "g":
        return 1 - 2 * s * e - e * e
    return e + s - 1


@pytest.mark.parametrize("name", ["f", "g", "h"])
def test_series_branch_meets_closed_form(orc, name):
    """The Taylor branch (s < 1) and the closed form (s >= 1) agree across
    the switch, where both are accurate to ~1e-15."""
    fn = getattr(orc.lib(), "orc_%ss" % name)
    for s in (1.0 - 1e-13, 0.999, 0.9, 0.75):
        assert fn(s) == pytest.approx(_closed(name, s), rel=2e-14, abs=0)
    assert fn(1.0 - 1e-15) == pytest.approx(fn(1.0), rel=1e-13, abs=0)


@pytest.mark.parametrize("name", ["f", "g", "h"])
def test_series_branch_small_arguments(orc, name):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    fn = getattr(orc.lib(), "orc_%ss" % name)
    for s in (1e-9, 1e-6, 1e-3, 0.05, 0.3):
        S = mp.mpf(s)
        e = mp.e ** (-S)
        ref = {"f": 2 * (e - 1) + S * (e + 1), "g": 1 - 2 * S * e - e * e, "h": e + S - 1}[name]
        assert fn(s) == pytest.approx(float(ref), rel=1e-14, abs=0)


def test_unconditioned_variance_identity(orc):
    """E[d^2] + Var(a) over v' ~ N(mu, sigma^2) equals the unconditioned
    variance 2 sigma^2/R^2 (s - 1 + e^{-s}) of the kinetic displacement."""
    L = orc.lib()
    R, mu, sigma = 3.0, 0.2, 1.7
    for theta in (0.01, 0.3, 2.0):
        s = R * theta
        # a and d^2 are affine / quadratic in (v' - mu): moments from three points
        a1 = L.orc_advection(R, mu, theta, mu + 1.0) - L.orc_advection(R, mu, theta, mu)
        d0 = L.orc_diffusion(R, mu, sigma, theta, mu) ** 2
        d1 = L.orc_diffusion(R, mu, sigma, theta, mu + 1.0) ** 2 - d0
        total = d0 + d1 * sigma ** 2 + a1 ** 2 * sigma ** 2
        assert total == pytest.approx(2 * sigma ** 2 / R ** 2 * (s - 1 + math.exp(-s)), rel=1e-12, abs=0)


def test_cosine_inverse_cdf(orc):
    L = orc.lib()
    from scipy import stats
    us = np.linspace(1e-6, 1.0, 2001)
    for u in us:
        x = L.orc_cosine_inverse(u)
        F = x + math.sin(2 * math.pi * x) / (2 * math.pi)
        assert 0.0 <= x < 1.0
        if u < 1.0:
            assert F == pytest.approx(u, abs=2e-15)
    rng = np.random.default_rng(5)
    xs = np.array([L.orc_cosine_inverse(u) for u in rng.random(20000)])
    cdf = lambda x: x + np.sin(2 * np.pi * x) / (2 * np.pi)
    assert stats.kstest(xs, cdf).pvalue > 1e-3


def test_cosine_inverse_near_the_centre(orc):
    """Near u = 1/2 the CDF is flat (F'(1/2) = 0), so F(x) = u cannot show an
    error in x there.  Compare x with the root of G(y) = y - sin(2 pi y)/(2 pi)
    = u - 1/2 solved in 60-digit arithmetic, and G itself with its closed form
    at small y, where the oracle sums its Taylor series."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    L = orc.lib()
    G = lambda y: y - mp.sin(2 * mp.pi * y) / (2 * mp.pi)
    for y in (1e-7, 1e-5, 1e-4, 1e-3, 0.01, 0.1, -1e-4, -0.05):
        assert L.orc_cosine_G(y) == pytest.approx(float(G(mp.mpf(y))), rel=1e-14, abs=0)
    for g in (1e-15, 1e-12, 1e-9, 1e-6, 1e-3, 0.1, 0.3, 0.49):
        for sgn in (1.0, -1.0):
            u = 0.5 + sgn * g
            g_eff = mp.mpf(u) - mp.mpf("0.5")            # exact: u - 1/2 in binary
            y0 = mp.sign(g_eff) * mp.cbrt(6 * abs(g_eff) / (2 * mp.pi) ** 2)
            y = mp.findroot(lambda t: G(t) - g_eff, y0)
            assert abs(L.orc_cosine_inverse(u) - float(mp.mpf("0.5") + y)) <= 3e-16, (u, y)
