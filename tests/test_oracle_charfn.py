"""The oracle's path law against the exact characteristic function of the KD
scheme (CPU only).

`kd_charfn.kd_charfn` computes phi_l(k) = E[cos(k D)] of one level's
displacement D by closed-form Gaussian integrals over the velocities and chi,
plus a dynamic program over the exponential flights (Alg. 1 with eqs.
advection and diffusion, Sec. 2).  It is checked here on its own (second
moment, ballistic limit, quadrature convergence).  Then it fixes, with no
other implementation of the scheme involved:

* E[cos k x_l(T)] of the fine path of every level (x_0 = 0);
* E[cos k x_{l-1}(T)] of the coarse path of a level-l pair.  In the
  homogeneous case the coarse path has the law of a single-level run at
  dt_{l-1} (Sec. 3.2), so this is phi_{l-1}(k);
* E[cos k x_l - cos k x_{l-1}] = phi_l(k) - phi_{l-1}(k).  The coupling makes
  this difference far less noisy than either term, so it is resolved to many
  standard errors;
* for the periodic problem (x_0 ~ 1 + cos 2 pi x, F(x) = (x mod 1)^2):
  E[F(x_l)] = 1/3 + phi_l(2 pi)/(2 pi^2), E[Y_l] = (phi_l - phi_{l-1})(2 pi)/(2 pi^2),
  and bin b of an nb-bin histogram holds the mass
  1/nb + phi_l(2 pi) (sin(2 pi (b+1)/nb) - sin(2 pi b/nb))/(2 pi).
  This pins the value of int x^2 f that the periodic benchmark estimates
  (eq. mlmc-compact), which has no closed form.
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle.kd_charfn import kd_charfn

Z = 4.5          # standard errors allowed per comparison
KS = (math.pi, 2 * math.pi, 4 * math.pi)

# (eps, T, dt0): kinetic (R dt0 = 0.1), mixed (R dt0 = 1) and near-diffusive
# (R dt0 = 5); levels 0..3 halve dt.
REGIMES = [(1.0, 0.2, 0.1), (0.1, 0.02, 0.01), (0.1, 0.05, 0.05)]


def msd(eps, T):
    return 2.0 * (T - eps * eps * (1.0 - math.exp(-T / (eps * eps))))


def second_moment(eps, dt, n, h=1e-3):
    """-phi''(0) by a Richardson-extrapolated difference of 2 (1 - phi(k))/k^2."""
    m = [2.0 * (1.0 - kd_charfn(k, eps, dt, n)) / (k * k) for k in (h, 2 * h)]
    return (4.0 * m[0] - m[1]) / 3.0


@pytest.mark.parametrize("eps,T,dt0", REGIMES + [(0.5, 0.5, 0.1), (2.0, 1.0, 0.25)])
def test_charfn_second_moment(eps, T, dt0):
    for level in (0, 2):
        dt = dt0 / 2 ** level
        n = int(round(T / dt))
        assert second_moment(eps, dt, n) == pytest.approx(msd(eps, T), rel=1e-6)


def test_charfn_ballistic_limit_and_quadrature():
    # R = 1e-6: a flight almost never ends before T, so D = sigma nu T.
    eps, T, k = 1e3, 1.0, 200 * math.pi
    sigma = 1.0 / eps
    assert kd_charfn(k, eps, 0.25, 4) == pytest.approx(math.exp(-0.5 * (k * sigma * T) ** 2),
                                                       rel=1e-5)
    assert kd_charfn(0.0, 0.1, 0.01, 4) == pytest.approx(1.0, abs=1e-15)
    for eps, dt, n in [(0.1, 0.05, 1), (0.1, 0.0125, 4), (1.0, 0.025, 8)]:
        a = kd_charfn(2 * math.pi, eps, dt, n, nodes=64)
        b = kd_charfn(2 * math.pi, eps, dt, n, nodes=96)
        assert abs(a - b) < 1e-11


def _check(emp, exact, what):
    emp = np.asarray(emp, np.float64)
    se = emp.std() / math.sqrt(emp.size)
    assert abs(emp.mean() - exact) <= Z * se + 1e-12, (what, emp.mean(), exact, se)


@pytest.mark.parametrize("eps,T,dt0", REGIMES)
def test_oracle_pairs_match_charfn(orc, eps, T, dt0):
    p = orc.Problem(eps=eps, T=T, dt0=dt0, M=2, L=3, seed=7)
    n = 400_000
    for level in range(4):
        xf, xc, _, _ = orc.pairs(p, level, 0, n, threads=8)
        for k in KS:
            pf = kd_charfn(k, eps, p.dt(level), p.nsteps(level))
            cf = np.cos(k * xf)
            _check(cf, pf, ("fine", level, k))
            if level == 0:
                continue
            pc = kd_charfn(k, eps, p.dt(level - 1), p.nsteps(level - 1))
            cc = np.cos(k * xc)
            _check(cc, pc, ("coarse", level, k))
            _check(cf - cc, pf - pc, ("difference", level, k))


def test_coupled_difference_is_resolved(orc):
    """The level-1 difference of the near-diffusive regime is tens of standard
    errors away from zero, so the pin above has teeth."""
    eps, T, dt0 = REGIMES[2]
    p = orc.Problem(eps=eps, T=T, dt0=dt0, M=2, L=1, seed=7)
    n = 400_000
    xf, xc, _, _ = orc.pairs(p, 1, 0, n, threads=8)
    d = np.cos(2 * math.pi * xf) - np.cos(2 * math.pi * xc)
    exact = kd_charfn(2 * math.pi, eps, p.dt(1), 2) - kd_charfn(2 * math.pi, eps, p.dt(0), 1)
    assert abs(exact) > 20 * d.std() / math.sqrt(n)


def periodic_exact(eps, dt, n):
    return 1.0 / 3.0 + kd_charfn(2 * math.pi, eps, dt, n) / (2 * math.pi ** 2)


def bin_masses(phi, nb):
    e = np.arange(nb + 1) / nb
    return 1.0 / nb + phi * np.diff(np.sin(2 * math.pi * e)) / (2 * math.pi)


def test_oracle_periodic_qoi_and_density_exact(orc):
    eps, T, dt0 = REGIMES[2]
    nb = 16
    p = orc.Problem(eps=eps, T=T, dt0=dt0, M=2, L=3, qoi=orc.QOI_X2_PERIODIC,
                    init=orc.INIT_COSINE, nbins=nb, lo=0.0, hi=1.0, seed=3)
    n = 400_000
    for level in range(4):
        s = orc.run_level(p, level, 0, n, threads=8)
        ef = periodic_exact(eps, p.dt(level), p.nsteps(level))
        se = math.sqrt((s.sqf2 / n - (s.sqf / n) ** 2) / n)
        assert abs(s.sqf / n - ef) <= Z * se, (level, s.sqf / n, ef, se)
        if level > 0:
            ec = periodic_exact(eps, p.dt(level - 1), p.nsteps(level - 1))
            se_y = math.sqrt(s.var() / n)
            assert abs(s.mean() - (ef - ec)) <= Z * se_y, (level, s.mean(), ef - ec, se_y)
        phi = kd_charfn(2 * math.pi, eps, p.dt(level), p.nsteps(level))
        expected = n * bin_masses(phi, nb)
        chi2 = float(np.sum((s.hist_f - expected) ** 2 / expected))
        assert stats.chi2.sf(chi2, nb - 1) > 1e-4, (level, chi2)


@pytest.mark.parametrize("eps,levels", [(1.0, (0, 1)), (0.1, (0, 1, 2))])
def test_oracle_periodic_benchmark_value(orc, eps, levels):
    """The periodic benchmark problem (T = 1, dt0 = 0.5): by T = 1 the cosine
    mode has decayed to phi(2 pi) = 4.9e-4 (level 0) and 2.2e-4 (level 1) at
    eps = 1, and below 1e-12 at eps = 0.1.  So int x^2 f = 1/3 + phi/(2 pi^2)
    is within 3e-5 of 1/3."""
    p = orc.Problem(eps=eps, T=1.0, dt0=0.5, M=2, L=max(levels), qoi=orc.QOI_X2_PERIODIC,
                    init=orc.INIT_COSINE, seed=4)
    n = 200_000
    for level in levels:
        exact = periodic_exact(eps, p.dt(level), p.nsteps(level))
        assert abs(exact - 1.0 / 3.0) < 3e-5
        s = orc.run_level(p, level, 0, n, threads=8)
        se = math.sqrt((s.sqf2 / n - (s.sqf / n) ** 2) / n)
        assert abs(s.sqf / n - exact) <= Z * se


def test_benchmark_exact_values_file():
    """tests/golden/periodic_benchmark_exact.json (read by the benchmark) holds
    what make_periodic_exact.py computes."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden",
                           "periodic_benchmark_exact.json")) as f:
        vals = {v["eps"]: v for v in json.load(f)["values"]}
    assert vals[1.0]["exact"] == pytest.approx(periodic_exact(1.0, 0.25, 4), rel=1e-15)
    for eps in (0.1, 1e-3):
        assert abs(vals[eps]["exact"] - 1.0 / 3.0) < 1e-12


def test_oracle_pairs_match_charfn_refinement_three(orc):
    """M = 3 (not a power of two): the coarse path of a level-l pair has the
    law of a single-level run at 3 dt_l."""
    eps, T, dt0 = 0.1, 0.045, 0.045          # R dt = 4.5, 1.5, 0.5
    p = orc.Problem(eps=eps, T=T, dt0=dt0, M=3, L=2, seed=8)
    n = 400_000
    for level in (1, 2):
        xf, xc, _, _ = orc.pairs(p, level, 0, n, threads=8)
        for k in KS:
            pf = kd_charfn(k, eps, p.dt(level), p.nsteps(level))
            pc = kd_charfn(k, eps, p.dt(level - 1), p.nsteps(level - 1))
            cf, cc = np.cos(k * xf), np.cos(k * xc)
            _check(cf, pf, ("fine", level, k))
            _check(cc, pc, ("coarse", level, k))
            _check(cf - cc, pf - pc, ("difference", level, k))
