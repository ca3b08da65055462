"""Heuristic level selection (Alg. 3) and estimates over a level set, CPU
only: the C ABI's mlkd_level_select and the oracle's restatement agree with
sets worked out by hand from the algorithm, and the oracle's gapped pairs
(coarsening M^gap) keep the properties of adjacent pairs."""
import math

import numpy as np
import pytest

CASES = [
    # V_l, Vd_l (Vd_0 unused) -> chosen levels
    # the homogeneous sketch: Vd rises above V, peaks, then decays like dt^3
    ([1.0] * 8, [0, 2.0, 3.0, 1.5, 0.9, 0.3, 0.05, 0.006], [3, 4, 5, 6, 7]),
    # decay already below V at level 1; slow decay skips levels
    ([1.0] * 6, [0, 0.5, 0.4, 0.3, 0.2, 0.05], [0, 1, 4, 5]),
    # L not reached by the halving rule is still appended
    ([1.0] * 6, [0, 0.5, 0.4, 0.3, 0.26, 0.26], [0, 1, 5]),
    # no level with Vd < V: a single-level estimate on L
    ([1.0] * 4, [0, 2.0, 2.0, 2.0], [3]),
    # the first level with Vd < V is L itself: the pair (L-1, L)
    ([1.0] * 4, [0, 2.0, 2.0, 0.5], [2, 3]),
]


@pytest.mark.parametrize("V,Vd,want", CASES)
def test_oracle_level_select(orc, V, Vd, want):
    assert orc.level_select(V, Vd) == want


@pytest.mark.parametrize("V,Vd,want", CASES)
def test_library_level_select_matches(V, Vd, want):
    from paper_2004_04071_gb300 import _build
    _build.build()
    import paper_2004_04071_gb300 as mk
    assert mk.level_select(V, Vd) == want


def test_gapped_pair_moments(orc):
    """A pair coupling level 4 with level 1 (M^gap = 8): both paths keep the
    closed-form second moment, and the coarse path has the law of the
    single-level scheme at level 1."""
    from scipy import stats
    p = orc.Problem(eps=0.2, T=1.0, dt0=0.5, M=2, L=4, level_set=[1, 4], seed=3)
    assert p.estimator_levels() == [(1, 2), (4, 8)]
    n = 100_000
    xf, xc, ef, ec = orc.pairs(p, 1, 0, n, threads=8)
    exact = 2.0 * (1.0 - 0.04 * (1.0 - math.exp(-1.0 / 0.04)))
    for x in (xf, xc):
        q = x * x
        assert abs(q.mean() - exact) < 4.5 * q.std() / math.sqrt(n)
    xs, _ = orc.single_paths(orc.Problem(eps=0.2, T=1.0, dt0=0.5, seed=99), 1, 0, 20_000)
    assert stats.ks_2samp(xc[:20_000], xs).pvalue > 1e-3
    # the fine path is the level-4 single path, bit for bit
    x4, _ = orc.single_paths(p, 4, 0, 1000)
    assert np.array_equal(xf[:1000], x4)


def test_level_set_estimate_telescopes(orc):
    p = orc.Problem(eps=0.3, T=0.5, dt0=0.1, M=2, L=4, level_set=[1, 2, 4], seed=5,
                    n_fixed=[60_000, 30_000, 20_000])
    r = orc.estimate(p, threads=8)
    exact = 2.0 * (0.5 - 0.09 * (1.0 - math.exp(-0.5 / 0.09)))
    assert [s.n for s in r.levels] == [60_000, 30_000, 20_000]
    assert abs(r.estimate - exact) < 4.5 * math.sqrt(r.variance)


# ---------------------------------------------------------------------------
# Level selection by optimisation (Sec. 4.2, eqs. level_selection, integerLP,
# V_approx).
# ---------------------------------------------------------------------------
def _lib():
    from paper_2004_04071_gb300 import _build
    _build.build()
    import paper_2004_04071_gb300 as mk
    return mk


def test_v_pair_approx_special_cases(orc):
    """eq. V_approx reduces to (sqrt V_i - sqrt V_j)^2 for perfectly
    correlated levels, to V_i + V_j where the bounds admit rho_{i,j} = 0, and
    to the exact Var(Q_L - Q_j) = V_L + V_j - 2 rho sqrt(V_L V_j) when one of
    the levels is L (rho_{L,L} = 1)."""
    assert orc.v_pair_approx(4.0, 1.0, 1.0, 1.0) == pytest.approx((2.0 - 1.0) ** 2)
    assert orc.v_pair_approx(4.0, 1.0, 0.6, 0.8) == pytest.approx(5.0)
    assert orc.v_pair_approx(4.0, 1.0, 0.3, 0.2) == pytest.approx(5.0)      # root argument < 0
    assert orc.v_pair_approx(4.0, 9.0, 1.0, 0.5) == pytest.approx(4.0 + 9.0 - 2 * 0.5 * 6.0)


def test_optimal_level_set_hand_example(orc):
    """L = 2, V = (1, 1, 1), C = (1, 4, 16), level 1 perfectly correlated
    with level 2, level 0 uncorrelated.  Costs worked by hand:
      {2}: sqrt(16) = 4;  {0,2}: 1 + sqrt(2 * 17);  {0,1,2}: 1 + sqrt(2 * 5) + 0;
      {1,2}: sqrt(4) + sqrt(0 * 20) = 2  (the optimum)."""
    V, rho, C = [1.0, 1.0, 1.0], [0.0, 1.0], [1.0, 4.0, 16.0]
    assert orc.level_set_cost([2], V, rho, C) == pytest.approx(4.0)
    assert orc.level_set_cost([0, 2], V, rho, C) == pytest.approx(1 + math.sqrt(34))
    assert orc.level_set_cost([0, 1, 2], V, rho, C) == pytest.approx(1 + math.sqrt(10))
    assert orc.level_set_cost([1, 2], V, rho, C) == pytest.approx(2.0)
    assert orc.level_select_opt(V, rho, C) == [1, 2]
    assert _lib().level_select_opt(V, rho, C) == [1, 2]


def test_library_optimal_selection_equals_brute_force(orc):
    """The library's shortest-path solution equals the oracle's enumeration
    of every subset on 300 random problems with L = 1..9, shaped like the
    homogeneous curves (variances and costs spanning decades)."""
    mk = _lib()
    rng = np.random.default_rng(11)
    for t in range(300):
        L = int(rng.integers(1, 10))
        V = list(10.0 ** rng.uniform(-3, 1, L + 1))
        C = sorted(10.0 ** rng.uniform(0, 4, L + 1))
        rho = list(rng.uniform(0.0, 1.0, L))
        assert mk.level_select_opt(V, rho, C) == orc.level_select_opt(V, rho, C), t


def test_level_pilot_statistics(orc):
    """Pilot of Sec. 4.2 on a small free-space problem: the level variances
    match those of plain single-level runs at each step size (same law),
    correlations lie in [-1, 1] and grow toward the finest level, and the
    cost per path does not fall as the step shrinks."""
    p = orc.Problem(eps=0.5, T=0.5, dt0=0.1, M=2, L=4, qoi=0, init=0, seed=3)
    V, rho, C = orc.level_pilot(p, 20000, threads=8)
    assert len(V) == 5 and len(rho) == 4 and len(C) == 5
    assert all(-1.0 <= r <= 1.0 for r in rho)
    assert rho[-1] > rho[0] and rho[-1] > 0.9
    assert all(b >= a - 1e-9 for a, b in zip(C[:-1], C[1:]))
    for i in (0, 2, 4):
        xs, es = orc.single_paths(orc.Problem(eps=0.5, T=0.5, dt0=0.1, M=2, L=4, seed=77), i, 0, 20000)
        vs = float(np.var(xs * xs, ddof=1))
        # x^2 has kurtosis near 26 here: each sample variance carries about 3.5 %
        assert abs(V[i] - vs) < 0.2 * vs


def test_warmup_tau_by_hand(orc):
    """Sec. 5.3: tau is the first level with dt_tau <= 1/R, else L."""
    P = lambda eps, L, dt0=0.5, M=2: orc.Problem(eps=eps, T=1.0, dt0=dt0, M=M, L=L)
    assert orc.warmup_tau(P(0.1, 8)) == 6          # R dt_l = 50 / 2^l: 0.78 at l = 6
    assert orc.warmup_tau(P(1.0, 1)) == 1          # R dt_1 = 0.25
    assert orc.warmup_tau(P(1e-3, 12)) == 12       # 5e5 / 2^12 > 1: none, so L
    assert orc.warmup_tau(P(0.1, 7)) == 6           # the level below L
    assert orc.warmup_tau(P(0.1, 5)) == 5           # 50 / 32 > 1; level 6 would qualify
    assert orc.warmup_tau(P(0.5, 4, dt0=1.0, M=4)) == 1    # R dt_1 = 4 * 1/4 = 1 exactly


def test_warmup_extrapolation_and_samples(orc):
    """Levels up to tau: sample variances of F(x_l) and Y_l over the first
    n_warmup pairs, recomputed here from the positions.  Past tau: V_l = V_tau,
    V_{l,l-1} = V_{tau,tau-1} M^(-3 (l - tau))."""
    p = orc.Problem(eps=0.2, T=1.0, dt0=0.5, M=2, L=7, seed=9)     # R dt_l = 12.5 / 2^l: tau = 4
    V, Vd, tau = orc.level_warmup(p, 300, threads=8)
    assert tau == 4 and Vd[0] == 0.0 and len(V) == len(Vd) == 8
    for l in range(tau + 1):
        xf, xc, _, _ = orc.pairs(p, l, 0, 300)
        assert V[l] == pytest.approx(np.var(xf ** 2, ddof=1), rel=1e-12, abs=0)
        if l:
            assert Vd[l] == pytest.approx(np.var(xf ** 2 - xc ** 2, ddof=1), rel=1e-12, abs=0)
    for l in range(tau + 1, 8):
        assert V[l] == V[tau]
        assert Vd[l] == pytest.approx(Vd[tau] / 8.0 ** (l - tau), rel=1e-15, abs=0)


def test_estimate_sequence_continues_one_estimator(orc, monkeypatch):
    """The on-line phase of Sec. 5.3 with stubbed levels (sample variance V_l
    and cost C_l exactly, for every pair range): stage r raises each level to
    the larger of its current count and the optimal count for tol_r, and no
    further."""
    V = [4.0, 1.0, 0.05, 0.002]
    C = [3.0, 10.0, 40.0, 160.0]
    tols = [0.05, 0.02, 0.01]

    def fake_run_level(problem, level, first, count, threads=1):
        # sum Y^2 over pairs [0, N) is V (N - 1) for every N: the sample
        # variance stays exactly V however the ranges are merged
        return orc.LevelSums(n=count, sy=0.0, sy2=V[level] * (count - (first == 0)),
                             events_f=int(C[level] * count), events_c=0)

    monkeypatch.setattr(orc, "run_level", fake_run_level)
    p = orc.Problem(eps=0.5, T=0.5, dt0=0.1, M=2, L=3, n_warmup=100)
    res = orc.estimate_sequence(p, tols)
    have = [100] * 4
    for tol, r in zip(tols, res):
        have = [max(h, t) for h, t in zip(have, orc.optimal_counts(V, C, tol))]
        assert [s.n for s in r.levels] == have


def test_estimate_sequence_single_tolerance_is_the_estimate(orc):
    p = orc.Problem(eps=0.5, T=0.5, dt0=0.1, M=2, L=2, tol=0.01, seed=12, nbins=12, lo=-2.0,
                    hi=2.0)
    (r,) = orc.estimate_sequence(p, [0.01], threads=8)
    e = orc.estimate(p, threads=8)
    assert [s.n for s in r.levels] == [s.n for s in e.levels]
    assert r.estimate == e.estimate and r.variance == e.variance
    assert np.array_equal(r.density, e.density)
    rs = orc.estimate_sequence(p, [0.03, 0.015, 0.01], threads=8)
    for tol, s in zip([0.03, 0.015, 0.01], rs):
        assert s.variance <= tol * tol / 2 * (1 + 1e-12)
    for a, b in zip(rs[:-1], rs[1:]):
        assert all(x.n <= y.n for x, y in zip(a.levels, b.levels))
