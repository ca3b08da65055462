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


def _check_level(orc, po, level, n, sg, pairs_g, pairs_o, precision, what):
    """Checks one level's FP32 sums (and histograms, if sg has them) against
    (1) the FP64 sums of the same kernel's per-pair output, within the
    compensated-sum bound, and exact FP32 bin decisions of those positions;
    (2) the oracle on the same 24-bit stream, within the bounds the per-pair
    bound implies (tests/fp32_bounds.py).  Returns the per-bin density
    allowance of this level against the oracle, in counts."""
    xf_g, xc_g, kf_g, kc_g = pairs_g
    xf_o, xc_o, kf_o, kc_o = pairs_o
    coupled = level > 0
    so = orc.level_sums(po, level, xf_o, xc_o, kf_o, kc_o)
    assert sg["n"] == n
    assert sg["events_f"] == int(kf_g.sum()) and sg["events_c"] == int(kc_g.sum())
    same = (kf_g == kf_o) & (kc_g == kc_o)
    flips = int(n - same.sum())
    assert flips <= MAX_FLIP_FRACTION * n, (what, level, flips)
    if flips == 0:
        assert sg["events_f"] == so.events_f and sg["events_c"] == so.events_c

    # 1. the reduction of the kernel's own pairs
    host, form, terms = B.host_level_sums(True, coupled, xf_g, xc_g, precision)
    for k in SUM_KEYS:
        comp = precision == 2 or k not in ("sy", "sy2")
        tol = form[k] + B.sum_error(terms[k], comp, n)
        assert abs(sg[k] - host[k]) <= tol, (what, level, k, sg[k], host[k], tol)
    lo, hi, nb = 0.0, 1.0, po.nbins
    bf = B.fp32_bins(xf_g, lo, hi, nb, True)
    hg = [np.bincount(bf[bf >= 0], minlength=nb), np.zeros(nb, np.int64), np.zeros(nb, np.int64)]
    if coupled:
        bc = B.fp32_bins(xc_g, lo, hi, nb, True)
        both = (bf == bc) & (bf >= 0)
        hg[1] = np.bincount(bc[bc >= 0], minlength=nb)
        hg[2] = np.bincount(bf[both], minlength=nb)
    if "hist_f" in sg:
        for got, want in zip((sg["hist_f"], sg["hist_c"], sg["hist_both"]), hg):
            assert np.array_equal(got, want), (what, level)

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
        print("%s level %d prec %d %s: |gpu - oracle| = %.3e, derived bound %.3e"
              % (what, level, precision, k, err, bound[k]))
        assert err <= bound[k], (what, level, k, err, bound[k])
    ev = kf_o + kc_o
    af, nf = B.edge_allowance(xf_o[same], B.pair_delta(xf_o[same], ev[same]), lo, hi, nb, True)
    ac, nc = (B.edge_allowance(xc_o[same], B.pair_delta(xc_o[same], ev[same]), lo, hi, nb, True)
              if coupled else (np.zeros(nb, np.int64), 0))
    print("%s level %d prec %d: %d flipped pairs; positions near a bin edge %d (fine) %d (coarse) "
          "of %d pairs" % (what, level, precision, flips, nf, nc, n))
    for x in (xf_o[~same], xf_g[~same], xc_o[~same], xc_g[~same]):
        b = B.fp32_bins(x, lo, hi, nb, True)
        np.add.at(af, b[b >= 0], 1)
        np.add.at(ac, b[b >= 0], 1)
    ho = (so.hist_f, so.hist_c, so.hist_both)
    assert np.all(np.abs(hg[0] - ho[0]) <= af), (what, level)
    assert np.all(np.abs(hg[1] - ho[1]) <= ac), (what, level)
    assert np.all(np.abs(hg[2] - ho[2]) <= af + ac), (what, level)
    return af + ac, hg


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("level", [0, 8])
def test_fp32_level_sums_and_histograms_against_oracle(orc, mk, ctx, level, precision):
    """The FP32 modes' level sums and histograms of the per-level form against
    the oracle on the same 24-bit stream, on the benchmark's periodic problem
    at eps = 0.1 (level 8: its busiest coupled level; level 0: single paths),
    2^17 pairs.  The per-pair output of the same kernel (mlkd_debug_pairs)
    gives the positions that feed the sums and histograms:

    1. Reduction: the kernel's sums against the FP64 sums of its own per-pair
       QoIs, within the compensated-sum bound; its histograms against the
       FP32 bin decisions of those positions, exactly.
    2. Oracle: each sum within the bound that the per-pair bound implies;
       each histogram bin within the count of pairs whose oracle position
       lies within the per-pair bound of that bin's edges.  Pairs whose event
       sequence differs (at most 1e-3 of them) enter with their actual
       difference."""
    d = W.periodic_problem(0.1)
    first, n = 12345, 1 << 17
    pg = gpu_problem(mk, d, precision=precision)
    po = oracle_problem(orc, d, recipe=orc.RECIPE_24)
    pairs_o = orc.pairs(po, level, first, n, threads=16)
    sg = ctx.run_level(pg, level, first, n)
    pairs_g = ctx.debug_pairs(pg, level, first, n)
    _check_level(orc, po, level, n, sg, pairs_g, pairs_o, precision, "per-level")


@pytest.mark.parametrize("precision", [1, 2])
def test_fp32_batched_step_against_oracle(orc, mk, precision):
    """The benchmark's batched kernel in its configuration (one pair per lane,
    unbounded slices, the CUDA graph, 128 bins) on the periodic problem at
    eps = 0.1 with fixed N_l (2^17 pairs on level 8, one round; 2*10^4 on the
    others).  For every level the batched kernel's own per-pair output
    (mlkd_debug_batch_pairs) is checked as in the per-level test: its sums
    against the FP64 sums of its pairs and, with its histograms, against the
    oracle on the same 24-bit stream; the density against both."""
    d = dict(W.periodic_problem(0.1), tol=0.0)
    L = d["L"]
    n_fixed = [20000] * L + [1 << 17]
    cfg = mk.batch_config(pairs_per_thread=1, substeps_per_launch=0, use_graph=1,
                          max_requests=16, max_nbins=128)
    po = oracle_problem(orc, d, recipe=orc.RECIPE_24)
    p = gpu_problem(mk, d, precision=precision, n_fixed=n_fixed)
    nb, h = d["nbins"], 1.0 / d["nbins"]
    c = mk.Context(0, arena_bytes=mk.batch_workspace_bytes(cfg))
    try:
        ref = c.estimate_batch([p], cfg)[0]
        dens_host = np.zeros(nb)
        dens_o = np.zeros(nb)
        allow = np.zeros(nb)
        for level in range(L + 1):
            n = n_fixed[level]
            r, *pairs_g = c.debug_batch_pairs(p, cfg, level)
            # the readout run is the benchmarked computation: same result
            assert r.estimate == ref.estimate and np.array_equal(r.density, ref.density)
            pairs_o = orc.pairs(po, level, 0, n, threads=16)
            a, hg = _check_level(orc, po, level, n, r.levels[level], tuple(pairs_g), pairs_o,
                                 precision, "batched")
            so = orc.level_sums(po, level, *pairs_o)
            dens_host += (hg[0] - hg[1]) / n / h
            dens_o += (so.hist_f - so.hist_c) / n / h
            allow += a / n / h
    finally:
        c.close()
    assert np.allclose(ref.density, dens_host, rtol=1e-12, atol=1e-12)
    err = np.abs(ref.density - dens_o)
    print("prec %d: density |gpu - oracle| max %.3e, allowance min %.3e"
          % (precision, err.max(), allow.min()))
    assert np.all(err <= allow + 1e-12 * np.abs(dens_o) + 1e-15)


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
