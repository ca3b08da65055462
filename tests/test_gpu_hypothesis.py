"""Sec. 5.1 consistency protocol on the GPU's own coarse random numbers
(GPU only).

The kernel's coarse steps are read out (mlkd_debug_coarse_draws): nu~ of
eq. nu-update, E~ = R tau~ of eq. epsilon-update and chi~ of eq. chi-update,
recorded for every collision of consecutive pairs until N = 1000 values are
available, as in the protocol.  The background is homogeneous with R = 1000
(the paper's b; its a = 0), T = 1, fine step dt_l = T/2^l and coarse step
M dt_l, i.e. the level set {l - log2 M, l}.

* FP64: the draws equal the oracle's (same pairs, same stream) to 1e-12.
* FP32: the Table hypothesis sweep -- l = 1..10, M in {2, 4, ..., 64} with
  M <= 2^l -- gives A^2 and p for each variable; the table is printed in
  the paper's layout.  With 135 tests at once the check is family-wise: every
  p above 0.01/135 (Bonferroni at 1 %), and the p-values themselves uniform
  (Kolmogorov-Smirnov p > 0.001), which a biased variable would break
  across its whole column.
"""
import math

import numpy as np
import pytest
from scipy import stats

from ad_test import ad_pvalue, ad_statistic
from helpers import gpu_problem, oracle_problem

pytestmark = pytest.mark.gpu

R = 1000.0
N = 1000


@pytest.fixture(scope="module")
def mk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_04071_gb300 as mk
    mk.lib()
    return mk


@pytest.fixture(scope="module")
def ctx(mk):
    c = mk.Context(0)
    yield c
    c.close()


def cell_problem(level, M, seed=0):
    """Level set {level - log2 M, level} on dt_l = 2^-l (dt0 = T = 1)."""
    m = int(round(math.log2(M)))
    return dict(eps=1.0 / math.sqrt(R), T=1.0, dt0=1.0, M=2, L=level, qoi=0, init=0, nbins=0,
                seed=seed, level_set=[level - m, level])


def gpu_draws(mk, ctx, d, precision, n_want=N, n_pairs=1000):
    # a pair has at most one coarse step per coarse grid step
    lo, hi = d["level_set"]
    per_pair = 2 ** lo + 8
    nu, E, chi, pair_of, counts = ctx.debug_coarse_draws(gpu_problem(mk, d, precision=precision),
                                                         1, 0, n_pairs, per_pair)
    # every pair must fit its coarse steps, so the concatenation is the
    # protocol's "all collisions of consecutive pairs"
    first_short = np.nonzero(counts > per_pair)[0]
    stop = first_short[0] if first_short.size else n_pairs
    keep = pair_of < stop
    assert keep.sum() >= n_want, (d, stop, keep.sum())
    return nu[keep][:n_want], E[keep][:n_want], chi[keep][:n_want], pair_of[keep][:n_want]


@pytest.mark.parametrize("level,M", [(1, 2), (3, 8), (5, 16), (6, 64), (8, 32)])
def test_fp64_coarse_draws_match_oracle(orc, mk, ctx, level, M):
    d = cell_problem(level, M, seed=3)
    nu, E, chi, pair_of = gpu_draws(mk, ctx, d, mk.PREC_FP64)
    last = int(pair_of[-1]) + 1
    nu_o, E_o, chi_o, pair_o = orc.coarse_draws(oracle_problem(orc, d), 1, 0, last, N)
    assert len(nu_o) == N and np.array_equal(pair_o, pair_of)
    for g, o in ((nu, nu_o), (E, E_o), (chi, chi_o)):
        assert np.all(np.abs(g - o) <= 1e-12 * np.maximum(1.0, np.abs(o)))


def test_table_hypothesis_on_gpu_draws(mk, ctx):
    cdfs = {"nu": stats.norm.cdf, "E": stats.expon.cdf, "chi": stats.norm.cdf}
    Ms = (2, 4, 8, 16, 32, 64)
    table = {}
    for level in range(1, 11):
        for M in Ms:
            if M > 2 ** level:
                continue
            nu, E, chi, _ = gpu_draws(mk, ctx, cell_problem(level, M), mk.PREC_FP32_COMP)
            for name, x in (("nu", nu), ("E", E), ("chi", chi)):
                a2 = ad_statistic(x, cdfs[name])
                table[(level, M, name)] = (a2, ad_pvalue(a2))
    lines = ["Table hypothesis layout (GPU FP32 draws, homogeneous R = 1000, N = 1000): A^2 p"]
    for level in range(1, 11):
        for name in ("nu", "E", "chi"):
            cells = ["%5.3f %5.3f" % table[(level, M, name)] if (level, M, name) in table
                     else " " * 11 for M in Ms]
            lines.append("l=%-2d %-3s | %s" % (level, name, " | ".join(cells)))
    print("\n".join(lines))
    p = np.array([v[1] for v in table.values()])
    n = len(p)
    assert n == 135
    print("tests %d, p < 0.01: %d (expected about %.1f), min p %.4f" % (n, int((p < 0.01).sum()),
                                                                    0.01 * n, p.min()))
    assert p.min() > 0.01 / n
    assert stats.kstest(p, "uniform").pvalue > 1e-3
