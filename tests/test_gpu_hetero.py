"""Heterogeneous backgrounds B1/B2 of Sec. 5 on the GPU against the oracle
(GPU only).

The paper's test case: x(0) = 1, T = 1, mu = 0, sigma = 1, QoI x(T), rate
R_1(x) = b (1 + a |x - 1|) or R_2(x) = b for x <= 1, b (1 + a (x - 1))
beyond.  Flights solve eq. intinv per linear piece, the coarse flight
follows eq. epsilon-update, Alg. 2 in its general form; the KD coefficients
are the homogeneous ones at the collision point's rate (a stand-in for the
corrected coefficients that the paper does not print).
"""
import math

import numpy as np
import pytest

import fp32_bounds as B
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


def case(bg, a, b, dt0=0.5, M=2, L=4, seed=0):
    return dict(eps=1.0, T=1.0, dt0=dt0, M=M, L=L, qoi=3, init=2, x0=1.0, nbins=16, lo=-1.0,
                hi=3.0, seed=seed, background=bg, bg_a=a, bg_b=b)


CASES = {
    "B1_a10_b100": case(1, 10.0, 100.0),
    "B1_a0p5_b3": case(1, 0.5, 3.0, seed=3),
    "B2_a20_b10": case(2, 20.0, 10.0, seed=5),
    "B2_a2_b1000_M4": case(2, 2.0, 1000.0, dt0=1.0, M=4, L=3, seed=7),
    "B1_a100_b1": case(1, 100.0, 1.0, seed=9),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_per_pair_parity(orc, mk, ctx, name):
    d = CASES[name]
    po = oracle_problem(orc, d)
    pg = gpu_problem(mk, d, precision=mk.PREC_FP64)
    for level in sorted({0, 1, d["L"]}):
        xf_o, xc_o, kf_o, kc_o = orc.pairs(po, level, 777, 3001, threads=16)
        xf, xc, kf, kc = ctx.debug_pairs(pg, level, 777, 3001)
        assert np.array_equal(kf, kf_o) and np.array_equal(kc, kc_o), (name, level)
        assert fp64_close(xf, xf_o).all() and fp64_close(xc, xc_o).all(), (
            name, level, np.max(np.abs(xf - xf_o)), np.max(np.abs(xc - xc_o)))


@pytest.mark.parametrize("name", ["B1_a10_b100", "B2_a20_b10"])
def test_fp64_level_sums_and_histograms(orc, mk, ctx, name):
    d = CASES[name]
    po = oracle_problem(orc, d)
    for level in (0, 2, d["L"]):
        so = orc.run_level(po, level, 11, 20000, threads=16)
        sg = ctx.run_level(gpu_problem(mk, d), level, 11, 20000)
        assert sg["n"] == so.n
        assert sg["events_f"] == so.events_f and sg["events_c"] == so.events_c
        for key in ("sy", "sy2", "sqf", "sqf2", "sqc", "sqc2"):
            ref = getattr(so, key)
            assert abs(sg[key] - ref) <= 1e-12 * (abs(ref) + so.n), key
        assert np.array_equal(sg["hist_f"], so.hist_f)
        assert np.array_equal(sg["hist_c"], so.hist_c)
        assert np.array_equal(sg["hist_both"], so.hist_both)


@pytest.mark.parametrize("precision", [1, 2])
def test_fp32_per_pair_bound(orc, mk, ctx, precision):
    """FP32 state against the oracle on the same 24-bit stream within the
    FP32 per-pair bound of the homogeneous path (C = 16); pairs whose event
    sequence differs stay rare."""
    for name in ("B1_a10_b100", "B2_a20_b10"):
        d = CASES[name]
        po = oracle_problem(orc, d, recipe=orc.RECIPE_24)
        pg = gpu_problem(mk, d, precision=precision)
        for level in (0, 1, d["L"]):
            xf_o, xc_o, kf_o, kc_o = orc.pairs(po, level, 0, 20000, threads=16)
            xf, xc, kf, kc = ctx.debug_pairs(pg, level, 0, 20000)
            same = (kf == kf_o) & (kc == kc_o)
            assert (~same).sum() <= 1e-3 * len(same)
            ev = kf_o + kc_o
            worst = 0.0
            for g, o in ((xf, xf_o), (xc, xc_o)):
                r = np.abs(g - o)[same] / (ev[same] + 1.0) / 2.0 ** -24 / np.maximum(1.0, np.abs(o[same]))
                worst = max(worst, r.max(initial=0.0))
            print("%s prec %d level %d: flips %d, worst C %.3f" % (name, precision, level,
                                                                  (~same).sum(), worst))
            assert worst <= B.FP32_C


def test_adaptive_estimate_matches_oracle(orc, mk, ctx):
    """The adaptive MLMC of Sec. 4.1 on B1 (a = 10, b = 100, tol 0.01): the
    same N_l in every round as the oracle's controller, and the same
    estimate to FP64 rounding."""
    d = dict(CASES["B1_a10_b100"], tol=0.01, L=3)
    ro = orc.estimate(oracle_problem(orc, d), threads=16)
    rg = ctx.estimate(gpu_problem(mk, d, precision=mk.PREC_FP64))
    assert [lv["n"] for lv in rg.levels] == [s.n for s in ro.levels]
    assert rg.estimate == pytest.approx(ro.estimate, rel=1e-11, abs=1e-13)
    assert rg.variance == pytest.approx(ro.variance, rel=1e-9)
    assert rg.variance <= 0.01 ** 2 / 2 * (1 + 1e-9)


def test_symmetric_background_mean_position_is_one(mk, ctx):
    """B1 is symmetric about x0 = 1: E[x(T)] = 1 on every level and the level
    differences have mean 0 (4.5 standard errors, 2^22 pairs, FP32)."""
    d = CASES["B1_a10_b100"]
    pg = gpu_problem(mk, d, precision=mk.PREC_FP32_COMP)
    n = 1 << 22
    for level in (0, 2, 4):
        s = ctx.run_level(pg, level, 0, n)
        mf = s["sqf"] / n
        vf = s["sqf2"] / n - mf * mf
        assert abs(mf - 1.0) < 4.5 * math.sqrt(vf / n)
        if level:
            my = s["sy"] / n
            vy = s["sy2"] / n - my * my
            assert abs(my) < 4.5 * math.sqrt(vy / n) + 1e-12


def test_a_zero_matches_the_homogeneous_path(mk, ctx):
    """a = 0 is the homogeneous background R = b, mu = 0, sigma = 1: the
    heterogeneous kernel's pairs equal the homogeneous oracle's (the oracle's
    homogeneous path takes R, mu and sigma directly) in event counts and to
    1e-12 in position."""
    import ctypes

    import oracle as O
    b = 7.0
    het = dict(eps=1.0, T=1.0, dt0=0.25, M=2, L=3, qoi=0, init=0, nbins=0, seed=2, background=1,
               bg_a=0.0, bg_b=b)
    P = lambda a_, t: a_.ctypes.data_as(ctypes.POINTER(t))
    for level in (0, 1, 3):
        xf_h, xc_h, kf_h, kc_h = ctx.debug_pairs(gpu_problem(mk, het), level, 0, 4000)
        d = O.LevelDesc()
        d.R, d.mu, d.sigma = b, 0.0, 1.0
        d.dt, d.n, d.M, d.level = 0.25 / 2 ** level, 4 * 2 ** level, 2, level
        d.init, d.recipe, d.seed, d.request, d.coupled = 0, O.RECIPE_53, 2, 0, 1 if level else 0
        xf, xc = np.zeros(4000), np.zeros(4000)
        ef, ec = np.zeros(4000, np.int64), np.zeros(4000, np.int64)
        assert O.lib().orc_pairs(ctypes.byref(d), 0, 4000, P(xf, ctypes.c_double),
                                 P(xc, ctypes.c_double), P(ef, ctypes.c_int64),
                                 P(ec, ctypes.c_int64)) == 0
        assert np.array_equal(kf_h, ef) and np.array_equal(kc_h, ec)
        assert fp64_close(xf_h, xf).all() and fp64_close(xc_h, xc).all()


BATCH_CASES = ["B1_a10_b100", "B2_a20_b10", "B2_a2_b1000_M4"]


@pytest.mark.parametrize("name", BATCH_CASES)
def test_batched_pairs_match_oracle_fp64(orc, mk, ctx, name):
    """The batched form runs the heterogeneous pairs one per lane, started
    from the warp's pool: every pair of every level is the oracle's (equal
    event counts, positions to 1e-12), and slicing the launch or another
    idle-lane threshold changes no pair."""
    d = CASES[name]
    n = 2001
    nf = [n] * (d["L"] + 1)
    pg = gpu_problem(mk, dict(d, n_fixed=nf), precision=mk.PREC_FP64)
    po = oracle_problem(orc, d)
    bctx = mk.Context(0, arena_bytes=mk.batch_workspace_bytes(mk.batch_config(max_requests=64,
                                                                                 max_nbins=128)))
    try:
        for level in sorted({0, 1, d["L"]}):
            xf_o, xc_o, kf_o, kc_o = orc.pairs(po, level, 0, n, threads=16)
            base = None
            for sl, rm in ((0, 0), (7, 1), (64, 32)):
                cfg = mk.batch_config(pairs_per_thread=2, substeps_per_launch=sl, max_requests=64,
                                      max_nbins=128, refill_min=rm)
                r, xf, xc, kf, kc = bctx.debug_batch_pairs(pg, cfg, level)
                assert np.array_equal(kf, kf_o) and np.array_equal(kc, kc_o), (name, level, sl)
                assert fp64_close(xf, xf_o).all() and fp64_close(xc, xc_o).all(), (name, level, sl)
                if base is None:
                    base = (xf, xc)
                else:
                    assert np.array_equal(xf, base[0]) and np.array_equal(xc, base[1])
    finally:
        bctx.close()


def test_batched_estimates_match_per_level_form(mk, ctx):
    """B1 and B2 estimated together in one batched call (FP64, adaptive): the
    same N_l in every level and the same estimates, to FP64 rounding of the
    sums, as the per-level form one problem at a time."""
    ds = [dict(CASES["B1_a10_b100"], tol=0.01, L=3, request=3),
          dict(CASES["B2_a20_b10"], tol=0.01, L=3, request=4, seed=0)]
    probs = [gpu_problem(mk, d, precision=mk.PREC_FP64) for d in ds]
    bctx = mk.Context(0, arena_bytes=mk.batch_workspace_bytes(mk.batch_config(max_requests=64,
                                                                                 max_nbins=128)))
    try:
        rb = bctx.estimate_batch(probs, mk.batch_config(max_requests=64, max_nbins=128))
    finally:
        bctx.close()
    for p, b in zip(probs, rb):
        r = ctx.estimate(p)
        assert [lv["n"] for lv in b.levels] == [lv["n"] for lv in r.levels]
        assert [lv["events_f"] for lv in b.levels] == [lv["events_f"] for lv in r.levels]
        assert b.estimate == pytest.approx(r.estimate, rel=1e-12, abs=1e-14)
        assert b.variance == pytest.approx(r.variance, rel=1e-9)


def test_batched_fp32_pairs_within_bound(orc, mk, ctx):
    """FP32 pairs of the batched form against the oracle on the 24-bit stream
    within the per-pair FP32 bound; pairs whose event sequence differs stay
    rare."""
    d = CASES["B2_a20_b10"]
    n = 20000
    nf = [n] * (d["L"] + 1)
    pg = gpu_problem(mk, dict(d, n_fixed=nf), precision=mk.PREC_FP32_COMP)
    po = oracle_problem(orc, d, recipe=orc.RECIPE_24)
    bctx = mk.Context(0, arena_bytes=mk.batch_workspace_bytes(mk.batch_config(max_requests=64,
                                                                                 max_nbins=128)))
    try:
        for level in (0, 2, d["L"]):
            _, xf, xc, kf, kc = bctx.debug_batch_pairs(pg, mk.batch_config(max_requests=64, max_nbins=128),
                                                      level)
            xf_o, xc_o, kf_o, kc_o = orc.pairs(po, level, 0, n, threads=16)
            same = (kf == kf_o) & (kc == kc_o)
            assert (~same).sum() <= 1e-3 * n
            ev = kf_o + kc_o
            for g, o in ((xf, xf_o), (xc, xc_o)):
                assert np.all(np.abs(g - o)[same] <= B.pair_delta(o, ev)[same])
    finally:
        bctx.close()


def test_mixed_batch_is_rejected(mk):
    """One batched call holds either homogeneous or heterogeneous problems."""
    het = gpu_problem(mk, dict(CASES["B1_a10_b100"], tol=0.01), precision=mk.PREC_FP64)
    hom = gpu_problem(mk, dict(eps=0.5, T=0.5, dt0=0.1, M=2, L=2, qoi=0, init=0, nbins=0, tol=0.01,
                               seed=0), precision=mk.PREC_FP64)
    bctx = mk.Context(0, arena_bytes=mk.batch_workspace_bytes(mk.batch_config(max_requests=64,
                                                                                 max_nbins=128)))
    try:
        with pytest.raises(mk.MlkdError):
            bctx.estimate_batch([het, hom], mk.batch_config(max_requests=64, max_nbins=128))
    finally:
        bctx.close()
