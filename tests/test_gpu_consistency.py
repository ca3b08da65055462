"""Statistical consistency of the CUDA path across level and coarsening
(GPU only).

* Sec. 5.1 protocol, swept over the refinement factor M and the level: the
  coarse path of a level-l pair (built by the Sec. 3 mapping and aggregation
  from the fine path's random numbers) has the law of an independent
  single-level run at dt_{l-1}, in position and in the mean number of
  collisions.  M runs from 2 to 64 (Sec. 5.1 uses M up to 64 as well).
* Sec. 5.2, homogeneous case: the variance of the level difference peaks near
  dt = 1/R and decays like dt^3 below it; the cost per pair grows like 1/dt
  above it and is flat below it.  Checked on the FP32 path.
"""
import math

import numpy as np
import pytest
from scipy import stats

from helpers import check_level_curve, gpu_problem, level_curve

pytestmark = pytest.mark.gpu


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


# (eps, M, level): kinetic, mixed and diffusive regimes at every coarsening.
SWEEP = [(0.2, 2, 1), (0.2, 2, 3), (0.2, 4, 1), (0.2, 4, 2), (0.2, 8, 1), (0.2, 8, 2),
         (0.2, 16, 1), (0.2, 16, 2), (0.2, 32, 1), (0.2, 64, 1), (0.2, 64, 2),
         (0.05, 4, 2), (0.05, 16, 1)]
# The 0.1 % critical value of each two-sample test keeps the family-wise
# false-rejection rate of the sweep near 1.3 % (13 cases).
ALPHA = 1e-3


@pytest.mark.parametrize("eps,M,level", SWEEP)
def test_coarse_path_law_matches_single_level(mk, ctx, eps, M, level):
    n = 20_000
    d = dict(eps=eps, T=1.0, dt0=0.5, M=M, L=level, qoi=0, init=0, nbins=0)
    _, xc, _, kc = ctx.debug_pairs(gpu_problem(mk, dict(d, seed=31), precision=mk.PREC_FP64),
                                   level, 0, n)
    xs, _, ks, _ = ctx.debug_pairs(gpu_problem(mk, dict(d, seed=977), precision=mk.PREC_FP64),
                                   level - 1, 0, n)
    ad = stats.anderson_ksamp([xc, xs])
    assert ad.statistic < ad.critical_values[-1], (ad.statistic, ad.critical_values[-1])
    assert stats.ks_2samp(xc, xs).pvalue > ALPHA
    kc = kc.astype(np.float64)
    ks = ks.astype(np.float64)
    assert abs(kc.mean() - ks.mean()) <= 5 * math.sqrt(kc.var() / n + ks.var() / n) + 1e-12


def test_level_variance_and_cost_curve_fp32(mk, ctx):
    eps = 0.1
    p = gpu_problem(mk, dict(eps=eps, T=1.0, dt0=0.5, M=2, L=12, qoi=0, init=0, nbins=0, seed=5),
                    precision=mk.PREC_FP32_COMP)

    def sums(level, n):
        st = ctx.run_level(p, level, 0, n)
        return st["sy"], st["sy2"], st["n"], st["events_f"] + st["events_c"]

    check_level_curve(level_curve(sums, 12, 100_000), 1.0 / eps ** 2)
