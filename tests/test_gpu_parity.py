"""Parity of the CUDA path with the oracle, through the C ABI (GPU only).

FP64 mode: every pair's final fine and coarse positions agree with the
oracle within 1e-12 * max(1, |x|) and the fine/coarse KD event counts agree
exactly, on the same Philox stream.  Level sums agree to 1e-12 relative to
the sum of magnitudes, histogram counts and event totals exactly.
"""
import math

import numpy as np
import pytest

import workloads as W
from helpers import fp64_close, gpu_problem, oracle_problem

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


REGIMES = {
    "two_level": dict(W.TWO_LEVEL, n_fixed=None),
    "diffusive": dict(eps=0.1, T=1.0, dt0=0.5, M=2, L=4, qoi=0, init=0, nbins=16, lo=-4.0, hi=4.0,
                      seed=3),
    "kinetic": dict(eps=2.0, T=1.0, dt0=0.25, M=2, L=3, qoi=0, init=0, nbins=0, seed=5),
    "M4_drift": dict(eps=0.3, T=0.5, dt0=0.25, M=4, L=2, qoi=0, init=0, nbins=0, seed=9, mu=0.7),
    "M8": dict(eps=0.05, T=1.0, dt0=0.5, M=8, L=2, qoi=0, init=0, nbins=0, seed=13),
    "periodic": dict(eps=0.1, T=1.0, dt0=0.5, M=2, L=5, qoi=1, init=1, nbins=128, lo=0.0, hi=1.0,
                     seed=21),
    "deep_diffusive": dict(eps=1e-3, T=1.0, dt0=0.5, M=2, L=6, qoi=1, init=1, nbins=64, lo=0.0,
                           hi=1.0, seed=2),
    # refinement factors that are not powers of two: the coarse step end is
    # found by division instead of a shift
    "M3": dict(eps=0.2, T=0.6, dt0=0.2, M=3, L=2, qoi=0, init=0, nbins=12, lo=-3.0, hi=3.0, seed=17),
    "M6_diffusive": dict(eps=0.05, T=1.0, dt0=0.5, M=6, L=2, qoi=1, init=1, nbins=0, seed=19),
    # the large refinement factors of the Sec. 5.1 sweep: windows of up to 64
    # fine steps per coarse step
    "M16": dict(eps=0.05, T=1.0, dt0=0.5, M=16, L=2, qoi=0, init=0, nbins=0, seed=29),
    "M32_periodic": dict(eps=0.1, T=1.0, dt0=1.0, M=32, L=2, qoi=1, init=1, nbins=32, lo=0.0,
                         hi=1.0, seed=31),
    "M64": dict(eps=0.02, T=0.5, dt0=0.5, M=64, L=2, qoi=0, init=0, nbins=0, seed=37),
}


def _compare_pairs(orc, mk, ctx, d, level, first, count, rel=1e-12):
    po = oracle_problem(orc, d)
    xf_o, xc_o, kf_o, kc_o = orc.pairs(po, level, first, count, threads=8)
    pg = gpu_problem(mk, d, precision=0)
    xf_g, xc_g, kf_g, kc_g = ctx.debug_pairs(pg, level, first, count)
    same_events = (kf_g == kf_o) & (kc_g == kc_o)
    assert same_events.all(), "event sequences differ for %d pairs" % (~same_events).sum()
    bad_f = ~fp64_close(xf_g, xf_o, rel)
    bad_c = ~fp64_close(xc_g, xc_o, rel)
    worst = max(np.max(np.abs(xf_g - xf_o) / np.maximum(1, np.abs(xf_o))),
                np.max(np.abs(xc_g - xc_o) / np.maximum(1, np.abs(xc_o))))
    assert not bad_f.any() and not bad_c.any(), "worst scaled error %.3g" % worst
    return worst


@pytest.mark.parametrize("name", sorted(REGIMES))
def test_fp64_per_pair_parity(orc, mk, ctx, name):
    d = REGIMES[name]
    for level in range(d["L"] + 1):
        # several tiles and a ragged tail, starting at an odd offset
        _compare_pairs(orc, mk, ctx, d, level, 777, 3001)


def test_fp64_parity_high_pair_index(orc, mk, ctx):
    """Pairs beyond 2^32 use the high counter word."""
    d = REGIMES["two_level"]
    _compare_pairs(orc, mk, ctx, d, 1, (1 << 33) + 5, 257)


def test_single_pair_and_empty(orc, mk, ctx):
    d = REGIMES["two_level"]
    _compare_pairs(orc, mk, ctx, d, 1, 0, 1)
    pg = gpu_problem(mk, d)
    st = ctx.run_level(pg, 1, 0, 0)
    assert st["n"] == 0 and st["sy"] == 0.0 and st["events_f"] == 0
    assert np.all(st["hist_f"] == 0)


def test_fp64_parity_at_the_largest_level(orc, mk, ctx):
    """2^30 fine steps (the FP64 cap), M = 4: kinetic pairs whose flights
    span hundreds of millions of steps, so step indices and flights in step
    units reach the top of their range."""
    d = dict(eps=0.5, T=1.0, dt0=1.0, M=4, L=15, qoi=0, init=0, nbins=0, seed=23)
    _compare_pairs(orc, mk, ctx, d, 15, 0, 300)
    _compare_pairs(orc, mk, ctx, d, 14, 1 << 20, 300)


def test_ballistic_pairs(orc, mk, ctx):
    d = dict(eps=1e4, T=1.0, dt0=0.5, M=2, L=2, qoi=0, init=0, nbins=0, seed=3)
    for level in (0, 1, 2):
        _compare_pairs(orc, mk, ctx, d, level, 0, 500)
    xf, xc, kf, kc = ctx.debug_pairs(gpu_problem(mk, d), 2, 0, 500)
    assert np.all(kf == 0) and np.all(kc == 0) and np.array_equal(xf, xc)


@pytest.mark.parametrize("name", ["two_level", "diffusive", "periodic"])
def test_level_sums_parity(orc, mk, ctx, name):
    d = REGIMES[name]
    for level in range(min(d["L"], 3) + 1):
        po = oracle_problem(orc, d)
        so = orc.run_level(po, level, 11, 20000, threads=8)
        sg = ctx.run_level(gpu_problem(mk, d), level, 11, 20000)
        assert sg["n"] == so.n
        assert sg["events_f"] == so.events_f and sg["events_c"] == so.events_c
        xf, xc, _, _ = orc.pairs(po, level, 11, 20000, threads=8)
        scale = np.sum(np.abs(orc.qoi_values(po, xf))) + np.sum(np.abs(orc.qoi_values(po, xc)))
        for key, ref in (("sy", so.sy), ("sqf", so.sqf), ("sqc", so.sqc)):
            assert abs(sg[key] - ref) <= 1e-12 * (scale + so.n), key
        for key, ref in (("sy2", so.sy2), ("sqf2", so.sqf2), ("sqc2", so.sqc2)):
            assert abs(sg[key] - ref) <= 1e-12 * (abs(ref) + scale * scale / max(so.n, 1) + so.n), key
        if d["nbins"]:
            assert np.array_equal(sg["hist_f"], so.hist_f)
            assert np.array_equal(sg["hist_c"], so.hist_c)
            assert np.array_equal(sg["hist_both"], so.hist_both)


def test_split_ranges_give_same_sums(mk, ctx):
    """Pair p always uses the same stream: two halves add up to the whole."""
    d = REGIMES["two_level"]
    pg = gpu_problem(mk, d)
    a = ctx.run_level(pg, 1, 0, 5000)
    b = ctx.run_level(pg, 1, 5000, 7000)
    w = ctx.run_level(pg, 1, 0, 12000)
    assert a["events_f"] + b["events_f"] == w["events_f"]
    assert math.isclose(a["sy"] + b["sy"], w["sy"], rel_tol=1e-12, abs_tol=1e-12)
    assert np.array_equal(a["hist_f"] + b["hist_f"], w["hist_f"])


def test_reproducible(mk, ctx):
    d = REGIMES["diffusive"]
    pg = gpu_problem(mk, d)
    a = ctx.run_level(pg, 3, 0, 50000)
    b = ctx.run_level(pg, 3, 0, 50000)
    assert a["sy"] == b["sy"] and a["sy2"] == b["sy2"] and a["events_c"] == b["events_c"]


@pytest.mark.parametrize("case", ["periodic_density", "hetero_B1"])
def test_estimate_reproducible(mk, ctx, case):
    """The adaptive per-level estimate runs the levels of each round at the
    same time on separate streams; the result, per-level sums and histograms
    included, is the same bit for bit from run to run (FP32 state)."""
    if case == "periodic_density":
        d = dict(eps=0.1, T=1.0, dt0=0.5, M=2, L=6, qoi=2, init=1, nbins=32, lo=0.0, hi=1.0,
                 tol=0.02, seed=4)
    else:
        d = dict(eps=1.0, T=1.0, dt0=1.0, M=2, L=8, qoi=3, init=2, x0=1.0, nbins=0, tol=1e-3,
                 seed=4, background=1, bg_a=10.0, bg_b=1000.0)
    pg = gpu_problem(mk, d, precision=mk.PREC_FP32_COMP)
    runs = [ctx.estimate(pg) for _ in range(3)]
    for r in runs[1:]:
        assert r.estimate == runs[0].estimate and r.variance == runs[0].variance
        assert r.levels == runs[0].levels
        if runs[0].density is not None:
            assert np.array_equal(r.density, runs[0].density)


def test_estimate_fixed_two_level(orc, mk, ctx):
    """The two-level free-space problem with N_0 = 10^4, N_1 = 2000."""
    d = dict(W.TWO_LEVEL)
    ro = orc.estimate(oracle_problem(orc, d), threads=8)
    rg = ctx.estimate(gpu_problem(mk, d))
    assert rg.levels[0]["n"] == 10_000 and rg.levels[1]["n"] == 2_000
    assert rg.estimate == pytest.approx(ro.estimate, rel=1e-12)
    assert rg.variance == pytest.approx(ro.variance, rel=1e-10, abs=0)
    np.testing.assert_allclose(rg.density, ro.density, rtol=1e-12, atol=1e-12)
    exact = W.msd_closed_form(d["eps"], d["T"])
    assert abs(rg.estimate - exact) < 4.5 * math.sqrt(rg.variance)


@pytest.mark.parametrize("qoi", [0, 2])
def test_estimate_adaptive_matches_oracle(orc, mk, ctx, qoi):
    if qoi == 0:
        d = dict(eps=0.5, T=0.5, dt0=0.1, M=2, L=3, qoi=0, init=0, nbins=0, tol=0.01,
                 n_warmup=100, seed=42)
    else:
        d = dict(eps=0.3, T=1.0, dt0=0.5, M=2, L=3, qoi=2, init=1, nbins=32, lo=0.0, hi=1.0,
                 tol=0.05, n_warmup=100, seed=43)
    ro = orc.estimate(oracle_problem(orc, d), threads=8)
    rg = ctx.estimate(gpu_problem(mk, d))
    n_o = [s.n for s in ro.levels]
    n_g = [lv["n"] for lv in rg.levels]
    assert n_g == n_o
    assert rg.estimate == pytest.approx(ro.estimate, rel=1e-11, abs=1e-13)
    assert rg.variance <= d["tol"] ** 2 / 2 * (1 + 1e-9)


def test_large_launch_sampled(orc, mk, ctx):
    """Full-wave launch (2^21 pairs on level 8 of the periodic eps = 0.1
    problem): a sample of pairs checked one by one against the oracle."""
    d = W.periodic_problem(0.1)
    level = 8
    n = 1 << 21
    xf, xc, kf, kc = ctx.debug_pairs(gpu_problem(mk, d), level, 0, n)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(n, 400, replace=False))
    po = oracle_problem(orc, d)
    for j in idx:
        a = orc.pairs(po, level, int(j), 1)
        assert kf[j] == a[2][0] and kc[j] == a[3][0]
        assert fp64_close(xf[j], a[0][0]) and fp64_close(xc[j], a[1][0])


@pytest.mark.parametrize("name", ["two_level", "diffusive", "periodic", "kinetic"])
def test_fp64_on_24bit_stream_matches_oracle(orc, mk, ctx, name):
    """FP64 state on the FP32 modes' random numbers against the oracle on the
    same 24-bit stream: the same 1e-12 bar as the FP64 mode."""
    d = REGIMES[name]
    for level in sorted({0, 1, d["L"]}):
        po = oracle_problem(orc, d, recipe=orc.RECIPE_24)
        xf_o, xc_o, kf_o, kc_o = orc.pairs(po, level, 5, 2000, threads=8)
        xf_g, xc_g, kf_g, kc_g = ctx.debug_pairs(gpu_problem(mk, d, precision=mk.PREC_FP64_U24),
                                                 level, 5, 2000)
        assert np.array_equal(kf_g, kf_o) and np.array_equal(kc_g, kc_o)
        assert fp64_close(xf_g, xf_o).all() and fp64_close(xc_g, xc_o).all()


def test_level_set_pairs_and_estimate(orc, mk, ctx):
    """Estimator levels coupling non-adjacent levels (Sec. 4.2): per pair and
    as a fixed-count estimate, against the oracle."""
    d = dict(eps=0.2, T=1.0, dt0=0.5, M=2, L=6, qoi=1, init=1, nbins=32, lo=0.0, hi=1.0, seed=8,
             level_set=[1, 2, 4, 6], n_fixed=[40000, 20000, 8000, 3000])
    po = oracle_problem(orc, d)
    po.level_set = d["level_set"]
    pg = mk.make_problem(precision=0, **{k: v for k, v in d.items()})
    for j in range(4):
        a = orc.pairs(po, j, 0, 1500, threads=8)
        b = ctx.debug_pairs(pg, j, 0, 1500)
        assert np.array_equal(b[2], a[2]) and np.array_equal(b[3], a[3])
        assert fp64_close(b[0], a[0]).all() and fp64_close(b[1], a[1]).all()
    ro = orc.estimate(po, threads=8)
    rg = ctx.estimate(pg)
    assert [lv["n"] for lv in rg.levels] == d["n_fixed"]
    assert rg.estimate == pytest.approx(ro.estimate, rel=1e-12)
    np.testing.assert_allclose(rg.density, ro.density, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("d", [
    dict(eps=0.5, T=0.5, dt0=0.1, M=2, L=4, qoi=0, init=0, nbins=0, seed=3),
    dict(eps=0.1, T=1.0, dt0=0.5, M=2, L=7, qoi=1, init=1, nbins=0, seed=12),
])
def test_level_pilot_matches_oracle(orc, mk, ctx, d):
    """Sec. 4.2 pilot on the GPU (FP64) against the oracle's on the same
    streams: V, rho and C per level within 1e-9, hence the same optimal level
    set."""
    po = oracle_problem(orc, d)
    Vo, ro, Co = orc.level_pilot(po, 3000, threads=8)
    Vg, rg, Cg = ctx.level_pilot(gpu_problem(mk, d, precision=mk.PREC_FP64), 3000)
    np.testing.assert_allclose(Vg, Vo, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(rg, ro, rtol=1e-9, atol=1e-9)
    assert Cg == Co
    assert mk.level_select_opt(Vg, rg, Cg) == orc.level_select_opt(Vo, ro, Co)


def test_level_warmup_matches_oracle(orc, mk, ctx):
    """Sec. 5.3 off-line phase on the device: tau, the sampled variances up
    to tau, the extrapolated ones past it, and the level set Alg. 3 picks."""
    for d in (dict(eps=0.2, T=1.0, dt0=0.5, M=2, L=7, qoi=0, init=0, nbins=0, seed=9),
              dict(eps=0.1, T=1.0, dt0=0.5, M=2, L=8, qoi=1, init=1, nbins=0, seed=3)):
        V, Vd, tau = ctx.level_warmup(gpu_problem(mk, d), 100)
        Vo, Vdo, tau_o = orc.level_warmup(oracle_problem(orc, d), 100, threads=8)
        assert tau == tau_o
        assert np.allclose(V, Vo, rtol=1e-9, atol=0) and np.allclose(Vd, Vdo, rtol=1e-9, atol=0)
        assert mk.level_select(V, Vd) == orc.level_select(Vo, Vdo)


@pytest.mark.parametrize("name", ["two_level", "periodic"])
def test_estimate_sequence_matches_oracle(orc, mk, ctx, name):
    """Sec. 5.3 on-line phase: one estimate continued through a decreasing
    tolerance sequence picks the oracle's N_l at every stage."""
    d = dict(REGIMES[name], L=3)
    tols = [0.02, 0.01, 0.005] if name == "two_level" else [0.004, 0.002]
    rg = ctx.estimate_sequence(gpu_problem(mk, d), tols)
    ro = orc.estimate_sequence(oracle_problem(orc, d), tols, threads=8)
    for tol, g, o in zip(tols, rg, ro):
        assert [lv["n"] for lv in g.levels] == [s.n for s in o.levels]
        assert g.estimate == pytest.approx(o.estimate, rel=1e-11, abs=1e-14)
        assert g.variance == pytest.approx(o.variance, rel=1e-9, abs=0)
        assert g.variance <= tol * tol / 2 * (1 + 1e-9)
        if d.get("nbins", 0) > 0:
            assert np.allclose(g.density, o.density, rtol=1e-11, atol=1e-12)
