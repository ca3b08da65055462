"""Statistical pins of the oracle (CPU only).

* Mean-square displacement: for the homogeneous background the KD scheme
  reproduces the first two moments of the kinetic process at every step size
  (a and d are the exact conditional mean and spread, Sec. 2), so
  E[x(T)^2] = mu^2 T^2 + 2 sigma^2/R^2 (RT - 1 + e^{-RT}); with R = 1/eps^2 and
  sigma = 1/eps this is 2(T - eps^2(1 - e^{-T/eps^2})).  This holds for the
  fine and for the coarse path of every pair, so E[Y_l] = 0 for F = x^2.
* Brownian limit eps -> 0: x(T) ~ N(0, 2T).
* Coarse random numbers: nu~ ~ N(0,1), E~ ~ Exp(1), chi~ ~ N(0,1) (Sec. 3.2,
  tested as in Sec. 5.1 with the Anderson-Darling statistic).
* Coarse law: x_{l-1}(T) of a pair has the law of an independent single-level
  run at dt_{l-1} (two-sample tests).
* Telescoping (eq. telsum): sum of level means = finest-level mean.
* Sample counts (eqs. Nopt1/Noptj) and the MLMC error bound (eq. mse).
* Shape of the level-difference variance and cost in the homogeneous case
  (Sec. 5.2): V_{l,l-1} grows as dt_l shrinks until a maximum near
  dt_l = 1/R, then decays like dt_l^3; C_{l,l-1} grows linearly with 1/dt_l
  until that point and is flat beyond it.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

from ad_test import ad_pvalue, ad_statistic
from helpers import check_level_curve, level_curve


def msd(eps, T, mu=0.0):
    return mu * mu * T * T + 2.0 * (T - eps * eps * (1.0 - math.exp(-T / (eps * eps))))


def test_ad_pvalues_reproduce_the_papers_table():
    """The AD p-value of tests/ad_test.py against (A^2, p) pairs printed in
    Table hypothesis (Sec. 5.1), to the printed three decimals; and the
    classic asymptotic percentage points 1.933 (10 %), 2.492 (5 %)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "ad_table_hypothesis.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) >= 8
    for level, M, var, a2, p in rows:
        assert abs(ad_pvalue(float(a2)) - float(p)) <= 1.5e-3, (level, M, var, a2, p)
    assert abs(ad_pvalue(1.933) - 0.10) < 2e-4
    assert abs(ad_pvalue(2.492) - 0.05) < 2e-4
    # the statistic itself: a sample at the quantiles (i - 1/2)/N of its own
    # law is nearly perfect (A^2 of order 1/N); the same sample shifted by
    # 0.2 is rejected outright
    N = 1000
    x = stats.norm.ppf((np.arange(1, N + 1) - 0.5) / N)
    assert 0.0 < ad_statistic(x, stats.norm.cdf) < 2.0 / N
    assert ad_pvalue(ad_statistic(x + 0.2, stats.norm.cdf)) < 1e-4


# Asymptotic critical values of A^2 for a fully specified law: 1 % -> 3.857,
# 0.1 % -> 5.973.  The paper rejects at p < 0.01 per test (Sec. 5.1); the
# parametrised test below runs 30 such tests, so each uses the 0.1 % value to
# keep the family-wise false-rejection rate near 3 %.
AD_CRIT_01PCT = 5.973


@pytest.mark.parametrize("eps,T,dt0,levels", [
    (0.5, 0.5, 0.1, (0, 1, 2, 3)),      # the 2-level free-space configuration, R dt = 0.4 .. 0.05
    (0.1, 1.0, 0.5, (0, 2, 4)),         # diffusive, R dt = 50 .. 3
    (2.0, 1.0, 0.25, (0, 1, 3)),        # kinetic, R dt = 0.06 ..
])
def test_second_moment_closed_form(orc, eps, T, dt0, levels):
    p = orc.Problem(eps=eps, T=T, dt0=dt0, M=2, L=max(levels), seed=21)
    exact = msd(eps, T)
    n = 200_000
    for level in levels:
        xf, xc, _, _ = orc.pairs(p, level, 0, n, threads=8)
        for x in ([xf] if level == 0 else [xf, xc]):
            q = x * x
            assert abs(q.mean() - exact) < 4.5 * q.std() / math.sqrt(n), (level, q.mean(), exact)


def test_first_and_second_moment_with_drift(orc):
    eps, T, mu = 0.4, 0.5, 1.3
    p = orc.Problem(eps=eps, T=T, dt0=0.25, M=2, L=2, seed=5, mu=mu)
    n = 200_000
    for level in (0, 2):
        xf, xc, _, _ = orc.pairs(p, level, 0, n, threads=8)
        for x in ([xf] if level == 0 else [xf, xc]):
            assert abs(x.mean() - mu * T) < 4.5 * x.std() / math.sqrt(n)
            q = x * x
            assert abs(q.mean() - msd(eps, T, mu)) < 4.5 * q.std() / math.sqrt(n)


def test_brownian_limit(orc):
    p = orc.Problem(eps=1e-4, T=1.0, dt0=0.5, M=2, L=2, seed=8)
    for level in (0, 2):
        xf, xc, _, _ = orc.pairs(p, level, 0, 20_000, threads=8)
        assert stats.kstest(xf / math.sqrt(2.0), "norm").pvalue > 1e-3
        if level:
            assert stats.kstest(xc / math.sqrt(2.0), "norm").pvalue > 1e-3


@pytest.mark.parametrize("eps,dt0,M,level", [(0.5, 0.1, 2, 1), (0.1, 0.5, 2, 4), (0.2, 0.5, 4, 2),
                                             (0.05, 0.5, 8, 2), (0.2, 0.5, 3, 2)])
def test_coarse_random_numbers_have_the_required_laws(orc, eps, dt0, M, level):
    """Sec. 5.1 protocol: A^2 of nu~, E~ and chi~ against their laws on
    N = 1000 draws (the paper's sample size) and on N = 20000."""
    p = orc.Problem(eps=eps, T=1.0, dt0=dt0, M=M, L=level, seed=4)
    nu_t, E_t, chi_t, _ = orc.coarse_draws(p, level, 0, 20000, 20000)
    assert len(nu_t) == 20000
    norm = stats.norm.cdf
    expo = stats.expon.cdf
    for N in (1000, 20000):
        sel = slice(0, N)
        assert ad_statistic(nu_t[sel], norm) < AD_CRIT_01PCT
        assert ad_statistic(E_t[sel], expo) < AD_CRIT_01PCT
        assert ad_statistic(chi_t[sel], norm) < AD_CRIT_01PCT


@pytest.mark.parametrize("eps,dt0,level", [(0.5, 0.1, 1), (0.2, 0.5, 3), (0.05, 0.5, 2)])
def test_coarse_path_law_matches_single_level(orc, eps, dt0, level):
    p = orc.Problem(eps=eps, T=1.0, dt0=dt0, M=2, L=level, seed=31)
    n = 20_000
    _, xc, _, ec = orc.pairs(p, level, 0, n, threads=8)
    q = orc.Problem(eps=eps, T=1.0, dt0=dt0, M=2, L=level, seed=977)
    xs, es = orc.single_paths(q, level - 1, 0, n)
    assert stats.ks_2samp(xc, xs).pvalue > 1e-3
    assert stats.anderson_ksamp([xc, xs]).pvalue > 1e-3
    # same number of coarse events on average as the coarse scheme itself
    assert abs(ec.mean() - es.mean()) <= 5 * math.sqrt(ec.var() / n + es.var() / n)


def test_telescoping_sum(orc):
    p = orc.Problem(eps=0.3, T=0.5, dt0=0.1, M=2, L=3, seed=17)
    n = 100_000
    total, var = 0.0, 0.0
    for level in range(4):
        s = orc.run_level(p, level, 0, n, threads=8)
        total += s.mean()
        var += s.var() / n
    q = orc.Problem(eps=0.3, T=0.5, dt0=0.1, M=2, L=3, seed=18)
    xf, _ = orc.single_paths(q, 3, 0, n)
    direct = np.mean(xf * xf)
    var += np.var(xf * xf) / n
    assert abs(total - direct) < 4.5 * math.sqrt(var)


def test_optimal_counts_formula(orc):
    # J = 1 reduces to N = 2 V / tol^2
    assert orc.optimal_counts([0.5], [3.0], 0.01) == [10000]
    # three levels, computed by hand from eqs. Nopt1/Noptj:
    # sum sqrt(V C) = 1 + 1 + 0.8 = 2.8; N_j = 200 sqrt(V_j/C_j) 2.8
    assert orc.optimal_counts([1.0, 0.25, 0.04], [1.0, 4.0, 16.0], 0.1) == [560, 140, 28]
    N = [560, 140, 28]
    assert sum(v / n for v, n in zip([1.0, 0.25, 0.04], N)) == pytest.approx(0.1 ** 2 / 2)


def test_mlmc_estimate_within_tolerance(orc):
    """Repeated adaptive estimates of E[x(T)^2]: empirical MSE below tol^2
    (bias is zero for this QoI)."""
    eps, T = 0.5, 0.5
    exact = msd(eps, T)
    tol = 0.02
    errs = []
    for seed in range(20):
        p = orc.Problem(eps=eps, T=T, dt0=0.1, M=2, L=2, tol=tol, seed=1000 + seed)
        r = orc.estimate(p, threads=8)
        assert r.variance <= tol * tol / 2 * 1.0000001
        errs.append(r.estimate - exact)
    mse = float(np.mean(np.square(errs)))
    # 20 draws of a variance <= tol^2/2: chi-square bound at the 0.1 % level
    assert mse < tol * tol / 2 * stats.chi2.ppf(0.999, 20) / 20


def test_periodic_qoi_identity(orc):
    """With x0 ~ 1 + cos(2 pi x) and a symmetric displacement D,
    E[(x(T) mod 1)^2] = 1/3 + E[cos(2 pi D)]/(2 pi^2)."""
    p = orc.Problem(eps=0.3, T=0.2, dt0=0.1, M=2, L=1, seed=2, init=orc.INIT_COSINE,
                    qoi=orc.QOI_X2_PERIODIC)
    n = 100_000
    xf, _, _, _ = orc.pairs(p, 0, 0, n, threads=8)
    L = orc.lib()
    x0 = np.array([L.orc_cosine_inverse(orc.stream_draws(p, 0, j, 1)[0][2]) for j in range(n)])
    D = xf - x0
    lhs = orc.qoi_values(p, xf)
    rhs = 1.0 / 3.0 + np.cos(2 * np.pi * D) / (2 * np.pi ** 2)
    diff = lhs - rhs
    assert abs(diff.mean()) < 4.5 * diff.std() / math.sqrt(n)


def test_density_counts_consistent(orc):
    p = orc.Problem(eps=0.5, T=0.5, dt0=0.1, M=2, L=1, nbins=20, lo=-3.0, hi=3.0, seed=0)
    xf, xc, ef, ec = orc.pairs(p, 1, 0, 5000)
    s = orc.level_sums(p, 1, xf, xc, ef, ec)
    inside_f = np.sum((xf >= -3) & (xf < 3))
    assert s.hist_f.sum() == inside_f
    assert np.all(s.hist_both <= np.minimum(s.hist_f, s.hist_c))
    # sum over pairs of Y_b^2 = f + c - 2 both >= |sum Y_b|
    assert np.all(s.hist_f + s.hist_c - 2 * s.hist_both >= np.abs(s.hist_f - s.hist_c))


@pytest.mark.parametrize("periodic", [False, True])
def test_density_variance_and_estimate_from_positions(orc, periodic):
    """The density QoI's V_l (largest bin variance of Y_b/h, the sup norm of
    R16) and the MLMC density estimate, recomputed by brute force from the
    pair positions: per-pair bin indicators and np.histogram, with no use of
    the oracle's counts or its bin function."""
    nb = 16
    if periodic:
        p = orc.Problem(eps=0.3, T=0.2, dt0=0.1, M=2, L=2, qoi=orc.QOI_DENSITY,
                        init=orc.INIT_COSINE, nbins=nb, lo=0.0, hi=1.0, seed=4,
                        n_fixed=[3000, 2000, 1000])
        lo, hi = 0.0, 1.0
        wrap = lambda x: x - np.floor(x)
    else:
        p = orc.Problem(eps=0.5, T=0.5, dt0=0.1, M=2, L=2, qoi=orc.QOI_DENSITY, nbins=nb,
                        lo=-1.5, hi=1.5, seed=4, n_fixed=[3000, 2000, 1000])
        lo, hi = -1.5, 1.5
        wrap = lambda x: x
    h = (hi - lo) / nb
    edges = lo + h * np.arange(nb + 1)

    def onehot(x):
        x = wrap(x)
        k = np.floor((x - lo) / h)
        inside = (x >= lo) & (x < hi)
        return (k[:, None] == np.arange(nb)[None, :]) & inside[:, None]

    dens = np.zeros(nb)
    for level, n in enumerate(p.n_fixed):
        xf, xc, ef, ec = orc.pairs(p, level, 0, n)
        s = orc.level_sums(p, level, xf, xc, ef, ec)
        yb = onehot(xf).astype(float) - (onehot(xc).astype(float) if level else 0.0)
        v_brute = np.var(yb, axis=0, ddof=1).max() / (h * h)
        assert orc.level_variance(p, s) == pytest.approx(v_brute, rel=1e-12, abs=0)
        hf = np.histogram(wrap(xf), bins=edges)[0]
        hc = np.histogram(wrap(xc), bins=edges)[0] if level else np.zeros(nb)
        dens += (hf - hc) / n / h
    r = orc.estimate(p)
    assert np.allclose(r.density, dens, rtol=1e-12, atol=1e-12)
    if periodic:
        assert np.sum(r.density) * h == pytest.approx(1.0, abs=1e-12)


def test_level_variance_and_cost_curve(orc):
    eps = 0.1
    p = orc.Problem(eps=eps, T=1.0, dt0=0.5, M=2, L=12, qoi=0, init=0, nbins=0, seed=5)

    def sums(level, n):
        s = orc.run_level(p, level, 0, n, threads=8)
        return s.sy, s.sy2, s.n, s.events_f + s.events_c

    check_level_curve(level_curve(sums, 12, 6000), 1.0 / eps ** 2)


def test_qoi_values_by_hand(orc):
    """F(x) = (x mod 1)^2 on the periodic interval and x^2 in free space, at
    points worked out by hand (negative x and whole periods included)."""
    per = orc.Problem(eps=1.0, T=1.0, dt0=0.5, qoi=orc.QOI_X2_PERIODIC, init=orc.INIT_COSINE)
    free = orc.Problem(eps=1.0, T=1.0, dt0=0.5)
    x = np.array([0.25, -0.25, 1.75, 3.0, -2.5, 0.0])
    assert np.array_equal(orc.qoi_values(per, x), [0.0625, 0.5625, 0.5625, 0.0, 0.25, 0.0])
    assert np.array_equal(orc.qoi_values(free, x), x * x)


@pytest.mark.parametrize("periodic,level", [(True, 0), (True, 2), (False, 1)])
def test_level_sums_from_positions(orc, periodic, level):
    """Every field of the oracle's level sums, its mean, sample variance and
    cost, recomputed with numpy from the pair positions and event counts; and
    sums of two pair ranges merged with add() equal the sums of their union."""
    if periodic:
        p = orc.Problem(eps=0.3, T=0.5, dt0=0.25, M=2, L=2, qoi=orc.QOI_X2_PERIODIC,
                        init=orc.INIT_COSINE, nbins=8, lo=0.0, hi=1.0, seed=6)
        F = lambda x: np.mod(x, 1.0) ** 2
    else:
        p = orc.Problem(eps=0.5, T=0.5, dt0=0.1, M=2, L=1, nbins=8, lo=-2.0, hi=2.0, seed=6)
        F = lambda x: x ** 2
    n, k = 6000, 2500
    xf, xc, ef, ec = orc.pairs(p, level, 0, n)
    s = orc.level_sums(p, level, xf, xc, ef, ec)
    qf = F(xf)
    qc = F(xc) if level else np.zeros(n)
    y = qf - qc
    close = lambda a, b: a == pytest.approx(b, rel=1e-12, abs=1e-300)
    assert s.n == n
    assert close(s.sy, y.sum()) and close(s.sy2, (y * y).sum())
    assert close(s.sqf, qf.sum()) and close(s.sqf2, (qf * qf).sum())
    assert close(s.sqc, qc.sum()) and close(s.sqc2, (qc * qc).sum())
    assert s.events_f == ef.sum() and s.events_c == ec.sum()
    assert close(s.mean(), y.mean()) and close(s.var(), np.var(y, ddof=1))
    assert close(s.cost(), (ef + ec).mean())
    a = orc.run_level(p, level, 0, k)
    a.add(orc.run_level(p, level, k, n - k))
    assert a.n == n and a.events_f == s.events_f and a.events_c == s.events_c
    for f in ("sy", "sy2", "sqf", "sqf2", "sqc", "sqc2"):
        assert close(getattr(a, f), getattr(s, f)), f
    for f in ("hist_f", "hist_c", "hist_both"):
        assert np.array_equal(getattr(a, f), getattr(s, f)), f


def test_controller_loop_reaches_its_targets(orc, monkeypatch):
    """The adaptive loop of Sec. 4.1 as a function of the level statistics.
    Levels are stubbed so that every pair range has sample variance V_l and
    cost C_l exactly.  After the warm-up the loop must raise each level to
    the count of eqs. Nopt1/Noptj, no further, and then stop."""
    V = [4.0, 1.0, 0.05, 0.002]
    C = [3.0, 10.0, 40.0, 160.0]
    tol = 0.01

    def fake_run_level(problem, level, first, count, threads=1):
        return orc.LevelSums(n=count, sy=0.0, sy2=V[level] * (count - 1),
                             events_f=int(C[level] * count), events_c=0)

    monkeypatch.setattr(orc, "run_level", fake_run_level)
    p = orc.Problem(eps=0.5, T=0.5, dt0=0.1, M=2, L=3, tol=tol, n_warmup=100)
    r = orc.estimate(p)
    want = [max(p.n_warmup, t) for t in orc.optimal_counts(V, C, tol)]
    assert [s.n for s in r.levels] == want


def test_bin_index_by_hand(orc):
    """Bins of [lo, hi): the lower edge belongs to bin 0, the upper edge is
    outside in free space, and a position just below hi whose (x - lo)/h rounds
    up to nb still lands in the last bin; periodic positions wrap first."""
    free = orc.Problem(eps=1.0, T=1.0, dt0=0.5, nbins=20, lo=-3.0, hi=3.0)
    below_hi = np.nextafter(3.0, 0.0)                  # (x - lo)/h rounds to 20.0
    x = np.array([-3.0, 3.0, below_hi, np.nextafter(-3.0, -4.0), 0.0, 2.95])
    assert list(orc.bin_index(free, x)) == [0, -1, 19, -1, 10, 19]
    per = orc.Problem(eps=1.0, T=1.0, dt0=0.5, nbins=8, qoi=orc.QOI_X2_PERIODIC,
                      init=orc.INIT_COSINE)
    x = np.array([1.0, -0.01, 0.5, 2.125, -3.9])
    assert list(orc.bin_index(per, x)) == [0, 7, 4, 1, 0]


def test_sample_variance_small_counts(orc):
    """Unbiased sample variance with the N - 1 divisor (R10) at N = 2 and 3,
    and 0 below two samples."""
    assert orc.LevelSums(n=2, sy=1.0, sy2=1.0).var() == 0.5          # samples {0, 1}
    assert orc.LevelSums(n=3, sy=3.0, sy2=5.0).var() == 1.0          # samples {0, 1, 2}
    assert orc.LevelSums(n=1, sy=2.0, sy2=4.0).var() == 0.0
