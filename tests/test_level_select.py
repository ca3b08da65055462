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
