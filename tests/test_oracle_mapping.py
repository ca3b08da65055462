"""Pins of the oracle's mapping and aggregation (Sec. 3, Alg. 2), CPU only.

* The kappa_k sequences printed with Fig. 2 (golden fixture).
* Homogeneous background: the coarse collision coincides with the fine
  collision kappa_k (eq. epsilon-update), so the coarse flight that starts at
  the coarse step end lasts exactly the remainder of the fine one.
* A particle that never collides before T moves ballistically on both levels:
  Y = 0 exactly.
* Hand traces of 3 particles over 4 fine steps, recomputed step by step in
  50-digit arithmetic from the KD step (Alg. 1) and the aggregation
  formulas of Sec. 3.2.
"""
import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _fig2_cases():
    with open(os.path.join(GOLDEN, "fig2_mapping.json")) as fh:
        return json.load(fh)["cases"]


@pytest.mark.parametrize("case", _fig2_cases(), ids=lambda c: c["name"])
def test_fig2_kappa_sequences(orc, case):
    flights = np.array(case["flights"])
    K = len(flights)
    R, dt, n, M = 1.0, 1.0, 4, 2
    rng = np.random.default_rng(1)
    nu = rng.standard_normal(K)
    chi = rng.standard_normal(K)
    out = orc.pair_injected(R, 0.0, 1.0, dt, n, M, 0.0, nu, flights * R, chi)
    # kappa_0 = 0 implicitly; one coarse step per recorded kappa
    assert [0] + list(out["kappa"]) == case["kappa"]
    # coarse collisions (before each coarse step) equal fine collisions kappa_k
    fine_coll = case["collisions"]
    kap = case["kappa"]
    for j, cc in enumerate(out["coarse_collision"]):
        assert cc == pytest.approx(fine_coll[kap[j]], abs=1e-15)
    # nu~_{k} = nu_{kappa_k}   (eq. nu-update)
    for j, k in enumerate(out["kappa"]):
        assert out["nu_t"][j] == nu[k]
    if "coarse_flight_1" in case:
        assert out["E_t"][0] / R == pytest.approx(case["coarse_flight_1"], abs=1e-15)
    # the fine path used one event per collision before T
    assert out["ev_f"] == len(fine_coll)


def test_no_collision_gives_zero_difference(orc):
    R, mu, sigma, dt, n, M = 3.0, 0.0, 2.0, 0.25, 8, 2
    nu0 = 0.731
    E0 = R * 5.0          # first flight 5 > T = 2
    out = orc.pair_injected(R, mu, sigma, dt, n, M, 0.125, [nu0], [E0], [])
    T = n * dt
    assert out["ev_f"] == 0 and out["ev_c"] == 0
    assert out["xf"] == out["xc"] == 0.125 + sigma * nu0 * T


def test_collision_on_grid_point_takes_full_diffusive_step(orc):
    """Reading 'floor+1': a collision exactly at a grid point starts a
    diffusive phase of one full step (eq. diffusive-time with mod = 0)."""
    R, dt, n = 2.0, 0.5, 4
    # flight of exactly 1 fine step: collision at t = 0.5, next phase at t = 1.0
    nu, E, chi = [0.3, -0.2], [R * 0.5, R * 10.0], [0.0]
    out = orc.pair_injected(R, 0.0, 1.0, dt, n, 2, 0.0, nu, E, chi, level=0)
    L = orc.lib()
    v0, v1 = nu[0], nu[1]
    a = L.orc_advection(R, 0.0, 0.5, v1)
    x_expect = v0 * 0.5 + a + v1 * (n * dt - 1.0)
    assert out["xf"] == pytest.approx(x_expect, rel=1e-14, abs=0)


def _hand_trace(flights, nu, chi, R, mu, sigma, dt, n, M):
    """Plain 50-digit evaluation of Alg. 2 for an injected stream, written
    from the KD step (Alg. 1: eqs. diffusive-time, advection, diffusion,
    position-update) and the aggregation of Sec. 3.2 (eqs. nu-update,
    epsilon-update, chi-update, zeta, tau', theta', alpha, beta)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    R, mu, sigma, dt = mp.mpf(R), mp.mpf(mu), mp.mpf(sigma), mp.mpf(dt)
    T = n * dt
    tau = [mp.mpf(f) for f in flights]

    def step_end(c, step):
        return (mp.floor(c / step) + 1) * step

    def kd(x, v, t, tau_k, v1, chi_k, step):
        c = t + tau_k
        theta = step_end(c, step) - c
        s = R * theta
        e = mp.e ** (-s)
        a = mu * theta + (v1 - mu) * (1 - e) / R
        d2 = (2 * sigma ** 2 / R ** 2 * (2 * (e - 1) + s * (e + 1))
              + (v1 - mu) ** 2 / R ** 2 * (1 - 2 * s * e - e * e))
        return x + v * tau_k + a + mp.sqrt(d2) * chi_k, step_end(c, step), theta

    # fine path (Alg. 1): phase starts, collisions and diffusive times
    starts, colls, thetas = [mp.mpf(0)], [], []
    xf, vf = mp.mpf(0), mu + sigma * nu[0]
    k = 0
    while True:
        c = starts[k] + tau[k]
        colls.append(c)
        if c >= T:
            break
        xf, t_new, theta = kd(xf, vf, starts[k], tau[k], mu + sigma * nu[k + 1], chi[k], dt)
        thetas.append(theta)
        starts.append(t_new)
        vf = mu + sigma * nu[k + 1]
        k += 1
    xf = xf + vf * (T - starts[k])

    zeta = lambda th: (1 - mp.e ** (-R * th)) / R

    def beta(th):
        tp = th - zeta(th)
        return mp.sqrt(2 * sigma ** 2 / R ** 2 * (mp.e ** (-R * tp) + R * tp - 1))

    # coarse path from the mapping (Sec. 3.1) and aggregation (Sec. 3.2)
    step_c = M * dt
    xc, vc, tc, tauc = mp.mpf(0), mu + sigma * nu[0], mp.mpf(0), tau[0]
    kappa = 0
    while tc + tauc < T:
        Ec = step_end(tc + tauc, step_c)
        m = kappa + 1
        while colls[m] < Ec:          # kappa_{k+1}: first later collision at/after Ec
            m += 1
        num = beta(thetas[kappa]) * chi[kappa]
        den = beta(thetas[kappa]) ** 2
        for j in range(kappa + 1, m):
            alpha = (tau[j] + zeta(thetas[j - 1])) * sigma
            b = beta(thetas[j])
            num += alpha * nu[j] + b * chi[j]
            den += alpha ** 2 + b ** 2
        chi_t = num / mp.sqrt(den)
        tau_t = colls[m] - Ec                     # homogeneous eq. epsilon-update
        xc, tc_new, _ = kd(xc, vc, tc, tauc, mu + sigma * nu[m], chi_t, step_c)
        vc, tc, tauc = mu + sigma * nu[m], tc_new, tau_t
        kappa = m
    xc = xc + vc * (T - tc)
    return float(xf), float(xc)


HAND = [
    # A: Fig. 2(a) flights, one collision per fine step
    dict(flights=[0.3, 0.1, 0.2, 0.3, 9.0], nu=[0.5, -1.2, 0.8, 0.1, -0.4], chi=[1.1, -0.3, 0.6, -0.9]),
    # B: Fig. 2(b) flights, an empty fine step
    dict(flights=[0.3, 1.5, 0.2, 9.0], nu=[-0.7, 0.2, 1.4, 0.9], chi=[0.4, -1.6, 0.05]),
    # C: first flight beyond T
    dict(flights=[9.0], nu=[1.3], chi=[]),
]


@pytest.mark.parametrize("case", HAND, ids=["A_fig2a", "B_fig2b", "C_ballistic"])
@pytest.mark.parametrize("R,mu,sigma", [(1.0, 0.0, 1.0), (2.5, 0.3, 1.7)])
def test_hand_traces(orc, case, R, mu, sigma):
    dt, n, M = 1.0, 4, 2
    flights = np.array(case["flights"])
    xf, xc = _hand_trace(case["flights"], case["nu"], case["chi"], R, mu, sigma, dt, n, M)
    out = orc.pair_injected(R, mu, sigma, dt, n, M, 0.0, case["nu"], flights * R,
                            case["chi"] + [0.0])
    assert out["xf"] == pytest.approx(xf, rel=1e-13, abs=1e-13)
    assert out["xc"] == pytest.approx(xc, rel=1e-13, abs=1e-13)


def test_fine_path_of_pair_equals_single_level_path(orc):
    """The coupling never perturbs the fine path: x_l of a level-l pair is
    the Alg. 1 path at dt_l on the same stream, bit for bit."""
    p = orc.Problem(eps=0.3, T=0.5, dt0=0.1, M=2, L=3, seed=11)
    for level in (1, 2, 3):
        xf, xc, ef, ec = orc.pairs(p, level, 100, 500)
        xs, es = orc.single_paths(p, level, 100, 500)
        assert np.array_equal(xf, xs)
        assert np.array_equal(ef, es)


def test_ballistic_limit_exact(orc):
    """R -> 0: no collision before T, x(T) = x0 + v0 T on every level."""
    p = orc.Problem(eps=1e4, T=1.0, dt0=0.5, M=2, L=2, seed=3)   # R = 1e-8
    for level in (0, 1, 2):
        xf, xc, ef, ec = orc.pairs(p, level, 0, 200)
        v0 = np.array([orc.stream_draws(p, level, j, 1)[0][0] for j in range(200)]) * p.sigma
        assert np.all(ef == 0)
        np.testing.assert_allclose(xf, v0 * p.T, rtol=1e-15)
        if level:
            assert np.array_equal(xf, xc)
