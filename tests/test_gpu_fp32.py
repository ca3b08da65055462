"""FP32 pair state against the oracle run on the same 24-bit-uniform stream
(GPU only).

The oracle computes in FP64 on the FP32 form of the Philox stream, so the
difference is the FP32 arithmetic of the pair kernel alone.  Per pair with
the same event sequence:
    |x_gpu - x_oracle| <= C * (events + 1) * 2^-24 * max(1, |x_oracle|)
with C = FP32_C below (measured on the two-level problem and the periodic
problem and fixed here).  Pairs whose event sequence differs (a floor of a
flight length that rounds across an integer in FP32) must be rare.
"""
import math

import numpy as np
import pytest

import workloads as W
from helpers import gpu_problem, oracle_problem

pytestmark = pytest.mark.gpu

FP32_C = 16.0
MAX_FLIP_FRACTION = 1e-3


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


CASES = {
    "two_level": dict(W.TWO_LEVEL, n_fixed=None),
    "periodic_eps0.1": W.periodic_problem(0.1),
    "diffusive_eps1e-3": dict(W.periodic_problem(1e-3), L=6),
    "kinetic": dict(eps=2.0, T=1.0, dt0=0.25, M=2, L=3, qoi=0, init=0, nbins=0, seed=5),
    "M3": dict(eps=0.2, T=0.6, dt0=0.2, M=3, L=2, qoi=0, init=0, nbins=0, seed=17),
    # 2^24 fine steps at level 12, the FP32 cap: step indices at the top of
    # the range where FP32 holds them exactly
    "largest_level": dict(eps=0.5, T=1.0, dt0=1.0, M=4, L=12, qoi=0, init=0, nbins=0, seed=23),
}


def _fp32_errors(orc, mk, ctx, d, level, precision, first=3, count=20000):
    po = oracle_problem(orc, d, recipe=orc.RECIPE_24)
    xf_o, xc_o, kf_o, kc_o = orc.pairs(po, level, first, count, threads=8)
    xf_g, xc_g, kf_g, kc_g = ctx.debug_pairs(gpu_problem(mk, d, precision=precision), level, first,
                                             count)
    same = (kf_g == kf_o) & (kc_g == kc_o)
    ev = (kf_o + kc_o + 1).astype(np.float64)
    rf = np.abs(xf_g - xf_o) / (ev * 2.0 ** -24 * np.maximum(1.0, np.abs(xf_o)))
    rc = np.abs(xc_g - xc_o) / (ev * 2.0 ** -24 * np.maximum(1.0, np.abs(xc_o)))
    return same, rf, rc


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("name", sorted(CASES))
def test_fp32_per_pair_bound(orc, mk, ctx, name, precision):
    d = CASES[name]
    worst = 0.0
    for level in sorted({0, 1, d["L"]}):
        same, rf, rc = _fp32_errors(orc, mk, ctx, d, level, precision)
        flips = 1.0 - same.mean()
        assert flips <= MAX_FLIP_FRACTION, (level, flips)
        w = max(rf[same].max(initial=0.0), rc[same].max(initial=0.0))
        worst = max(worst, w)
        print("%s prec=%d level=%d flips=%.2e worst C=%.3f p99 C=%.3f" %
              (name, precision, level, flips, w, np.percentile(np.r_[rf[same], rc[same]], 99)))
    assert worst <= FP32_C


@pytest.mark.parametrize("precision", [1, 2])
def test_fp32_level_sums_close_to_fp64(orc, mk, ctx, precision):
    """Per-level mean of Y_l in FP32 state versus the FP64 oracle: within the
    combined sampling error (same pairs, so much tighter in practice)."""
    d = dict(W.TWO_LEVEL, n_fixed=None)
    for level in (0, 1):
        so = orc.run_level(oracle_problem(orc, d), level, 0, 200000, threads=8)
        sg = ctx.run_level(gpu_problem(mk, d, precision=precision), level, 0, 200000)
        mo, mg = so.sy / so.n, sg["sy"] / sg["n"]
        vo = so.var()
        assert abs(mg - mo) < 3 * math.sqrt(vo / so.n) + 1e-6


def test_fp32_full_launch_sampled(orc, mk, ctx):
    """Full launch size of the benchmark's busiest coupled level (eps = 0.1,
    level 8, about 8e5 pairs): 400 sampled pairs against the oracle on the
    same 24-bit stream, one by one, within the FP32 bound."""
    d = W.periodic_problem(0.1)
    level, n = 8, 802_694
    xf, xc, kf, kc = ctx.debug_pairs(gpu_problem(mk, d, precision=mk.PREC_FP32_COMP), level, 0, n)
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(n, 400, replace=False))
    po = oracle_problem(orc, d, recipe=orc.RECIPE_24)
    flips = 0
    for j in idx:
        a = orc.pairs(po, level, int(j), 1)
        if kf[j] != a[2][0] or kc[j] != a[3][0]:
            flips += 1
            continue
        ev = a[2][0] + a[3][0] + 1
        for x, ref in ((xf[j], a[0][0]), (xc[j], a[1][0])):
            assert abs(x - ref) <= FP32_C * ev * 2.0 ** -24 * max(1.0, abs(ref))
    assert flips <= 1
