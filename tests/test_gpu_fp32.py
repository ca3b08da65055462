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

import fp32_bounds as B
import workloads as W
from helpers import gpu_problem, oracle_problem

pytestmark = pytest.mark.gpu

FP32_C = B.FP32_C
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


SUM_KEYS = ("sy", "sy2", "sqf", "sqf2", "sqc", "sqc2")


def _oracle_hist(orc, po, level, xf, xc):
    nb = po.nbins
    bf = orc.bin_index(po, xf)
    hf = np.bincount(bf[bf >= 0], minlength=nb)
    if level == 0:
        return hf, np.zeros(nb, np.int64), np.zeros(nb, np.int64)
    bc = orc.bin_index(po, xc)
    hc = np.bincount(bc[bc >= 0], minlength=nb)
    same = (bf == bc) & (bf >= 0)
    return hf, hc, np.bincount(bf[same], minlength=nb)


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("level", [0, 8])
def test_fp32_level_sums_and_histograms_against_oracle(orc, mk, ctx, level, precision):
    """The FP32 modes' level sums and histograms of the per-level form against
    the oracle on the same 24-bit stream, on the benchmark's periodic problem
    at eps = 0.1 (level 8: its busiest coupled level; level 0: single paths),
    2^17 pairs.

    1. Reduction: the kernel's sums against the FP64 sums of its own per-pair
       QoIs (the same kernel's per-pair output), within the compensated-sum
       bound; its histograms against the FP32 bin decisions of those
       positions, exactly.
    2. Oracle: each sum within the bound that the per-pair bound implies
       (tests/fp32_bounds.py); each histogram bin within the count of pairs
       whose oracle position lies within the per-pair bound of that bin's
       edges.  Pairs whose event sequence differs (none expected) enter with
       their actual difference."""
    d = W.periodic_problem(0.1)
    first, n = 12345, 1 << 17
    coupled = level > 0
    pg = gpu_problem(mk, d, precision=precision)
    po = oracle_problem(orc, d, recipe=orc.RECIPE_24)
    xf_o, xc_o, kf_o, kc_o = orc.pairs(po, level, first, n, threads=16)
    so = orc.level_sums(po, level, xf_o, xc_o, kf_o, kc_o)
    sg = ctx.run_level(pg, level, first, n)
    xf_g, xc_g, kf_g, kc_g = ctx.debug_pairs(pg, level, first, n)

    # counts
    assert sg["n"] == n
    assert sg["events_f"] == int(kf_g.sum()) and sg["events_c"] == int(kc_g.sum())
    same = (kf_g == kf_o) & (kc_g == kc_o)
    flips = int(n - same.sum())
    assert flips <= MAX_FLIP_FRACTION * n
    if flips == 0:
        assert sg["events_f"] == so.events_f and sg["events_c"] == so.events_c

    # 1. reduction of the kernel's own pairs
    host, form, terms = B.host_level_sums(True, coupled, xf_g, xc_g, precision)
    for k in SUM_KEYS:
        comp = precision == 2 or k not in ("sy", "sy2")
        tol = form[k] + B.sum_error(terms[k], comp, n)
        assert abs(sg[k] - host[k]) <= tol, (k, sg[k], host[k], tol)
    lo, hi, nb = 0.0, 1.0, pg.nbins
    bf = B.fp32_bins(xf_g, lo, hi, nb, True)
    hf = np.bincount(bf[bf >= 0], minlength=nb)
    assert np.array_equal(sg["hist_f"], hf)
    if coupled:
        bc = B.fp32_bins(xc_g, lo, hi, nb, True)
        assert np.array_equal(sg["hist_c"], np.bincount(bc[bc >= 0], minlength=nb))
        both = (bf == bc) & (bf >= 0)
        assert np.array_equal(sg["hist_both"], np.bincount(bf[both], minlength=nb))

    # 2. against the oracle
    bound = B.level_sum_bounds(True, coupled, xf_o[same], xc_o[same], kf_o[same], kc_o[same],
                               precision)
    if flips:
        _, _, tg = B.host_level_sums(True, coupled, xf_g[~same], xc_g[~same], precision)
        _, _, to = B.host_level_sums(True, coupled, xf_o[~same], xc_o[~same], precision)
        for k in SUM_KEYS:
            bound[k] += float(np.sum(np.abs(tg[k] - to[k]))) * (1 + 1e-6) + 1e-9
    for k in SUM_KEYS:
        err = abs(sg[k] - getattr(so, k))
        print("level %d prec %d %s: |gpu - oracle| = %.3e, derived bound %.3e"
              % (level, precision, k, err, bound[k]))
        assert err <= bound[k], (k, err, bound[k])
    ev = kf_o + kc_o
    ho = _oracle_hist(orc, po, level, xf_o, xc_o)
    af, nf = B.edge_allowance(xf_o, B.pair_delta(xf_o, ev), lo, hi, nb, True)
    ac, nc = (B.edge_allowance(xc_o, B.pair_delta(xc_o, ev), lo, hi, nb, True) if coupled
              else (np.zeros(nb, np.int64), 0))
    print("level %d prec %d: positions near a bin edge %d (fine) %d (coarse) of %d pairs"
          % (level, precision, nf, nc, n))
    if flips:
        extra = np.zeros(nb, np.int64)
        for x in (xf_o[~same], xf_g[~same], xc_o[~same], xc_g[~same]):
            b = B.fp32_bins(x, lo, hi, nb, True)
            np.add.at(extra, b[b >= 0], 1)
        af, ac = af + extra, ac + extra
    assert np.all(np.abs(sg["hist_f"].astype(np.int64) - ho[0]) <= af)
    assert np.all(np.abs(sg["hist_c"].astype(np.int64) - ho[1]) <= ac)
    assert np.all(np.abs(sg["hist_both"].astype(np.int64) - ho[2]) <= af + ac)


@pytest.mark.parametrize("precision", [1, 2])
def test_fp32_batched_step_against_oracle(orc, mk, precision):
    """The benchmark's batched form and configuration (one pair per lane,
    unbounded slices, the CUDA graph, 128 bins) on the periodic problem at
    eps = 0.1 with fixed N_l (2^17 pairs on level 8, one round, 2*10^4 on the
    others): every level's pair and event counts exactly, its six sums within
    the bound implied by the per-pair bound, and the density within the
    edge-count allowance of every level, all against the oracle on the same
    24-bit stream."""
    d = dict(W.periodic_problem(0.1), tol=0.0)
    L = d["L"]
    n_fixed = [20000] * L + [1 << 17]
    cfg = mk.batch_config(pairs_per_thread=1, substeps_per_launch=0, use_graph=1,
                          max_requests=16, max_nbins=128)
    c = mk.Context(0, arena_bytes=mk.batch_workspace_bytes(cfg))
    try:
        (rb,) = c.estimate_batch([gpu_problem(mk, d, precision=precision, n_fixed=n_fixed)], cfg)
    finally:
        c.close()
    po = oracle_problem(orc, d, recipe=orc.RECIPE_24)
    nb, lo, hi = d["nbins"], 0.0, 1.0
    h = (hi - lo) / nb
    dens_o = np.zeros(nb)
    dens_allow = np.zeros(nb)
    for level in range(L + 1):
        n = n_fixed[level]
        xf, xc, kf, kc = orc.pairs(po, level, 0, n, threads=16)
        so = orc.level_sums(po, level, xf, xc, kf, kc)
        lg = rb.levels[level]
        assert lg["n"] == n
        assert lg["events_f"] == so.events_f and lg["events_c"] == so.events_c, level
        bound = B.level_sum_bounds(True, level > 0, xf, xc, kf, kc, precision)
        for k in SUM_KEYS:
            err = abs(lg[k] - getattr(so, k))
            assert err <= bound[k], (level, k, err, bound[k])
        ev = kf + kc
        af, _ = B.edge_allowance(xf, B.pair_delta(xf, ev), lo, hi, nb, True)
        ac, _ = (B.edge_allowance(xc, B.pair_delta(xc, ev), lo, hi, nb, True) if level
                 else (np.zeros(nb, np.int64), 0))
        dens_o += (so.hist_f - so.hist_c) / n / h
        dens_allow += (af + ac) / n / h
    err = np.abs(rb.density - dens_o)
    print("prec %d: density |gpu - oracle| max %.3e, allowance min %.3e"
          % (precision, err.max(), dens_allow.min()))
    assert np.all(err <= dens_allow + 1e-12 * np.abs(dens_o) + 1e-15)


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
