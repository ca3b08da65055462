"""Batched form (one persistent pair kernel over a device work queue, rounds
scheduled per request on the device) against the per-level form and the
oracle (GPU only)."""
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
    cfg = mk.batch_config(max_requests=64, max_nbins=128)
    c = mk.Context(0, arena_bytes=mk.batch_workspace_bytes(cfg))
    yield c
    c.close()


def mixed_problems(precision, seed=5):
    return [
        dict(eps=0.5, T=0.5, dt0=0.1, M=2, L=3, qoi=0, init=0, nbins=0, tol=0.01, n_warmup=100,
             seed=seed, request=0),
        dict(eps=0.1, T=1.0, dt0=0.5, M=2, L=5, qoi=1, init=1, nbins=32, lo=0.0, hi=1.0, tol=0.003,
             n_warmup=100, seed=seed, request=1),
        dict(eps=2.0, T=1.0, dt0=0.25, M=2, L=2, qoi=0, init=0, nbins=0, tol=0.02, n_warmup=100,
             seed=seed, request=2),
        dict(eps=0.3, T=1.0, dt0=0.5, M=2, L=3, qoi=2, init=1, nbins=16, lo=0.0, hi=1.0, tol=0.05,
             n_warmup=100, seed=seed, request=3),
        dict(eps=1e-3, T=1.0, dt0=0.5, M=2, L=6, qoi=1, init=1, nbins=0, tol=0.003, n_warmup=100,
             seed=seed, request=4),
        dict(W.TWO_LEVEL, seed=seed, request=5),
        dict(eps=0.2, T=0.6, dt0=0.2, M=3, L=2, qoi=0, init=0, nbins=0, tol=0.01, n_warmup=100,
             seed=seed, request=6),
    ]


def test_batch_matches_per_level_fp64(mk, ctx):
    ds = mixed_problems(mk.PREC_FP64)
    probs = [gpu_problem(mk, d, precision=mk.PREC_FP64) for d in ds]
    cfg = mk.batch_config(max_requests=64, max_nbins=128)
    rb = ctx.estimate_batch(probs, cfg)
    for d, p, b in zip(ds, probs, rb):
        r = ctx.estimate(p)
        assert [lv["n"] for lv in b.levels] == [lv["n"] for lv in r.levels], d
        for lb, lr in zip(b.levels, r.levels):
            assert lb["events_f"] == lr["events_f"] and lb["events_c"] == lr["events_c"]
            assert lb["sy"] == pytest.approx(lr["sy"], rel=1e-12, abs=1e-12)
        assert b.estimate == pytest.approx(r.estimate, rel=1e-12, abs=1e-14)
        assert b.variance == pytest.approx(r.variance, rel=1e-10, abs=0)
        if p.nbins:
            np.testing.assert_allclose(b.density, r.density, rtol=1e-12, atol=1e-12)


def test_batch_fixed_counts_match_oracle(orc, mk, ctx):
    d = dict(W.TWO_LEVEL)
    ro = orc.estimate(oracle_problem(orc, d), threads=8)
    p = gpu_problem(mk, d, precision=mk.PREC_FP64)
    (rb,) = ctx.estimate_batch([p], mk.batch_config(max_requests=64, max_nbins=128))
    assert [lv["n"] for lv in rb.levels] == [10_000, 2_000]
    assert rb.estimate == pytest.approx(ro.estimate, rel=1e-12)
    np.testing.assert_allclose(rb.density, ro.density, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("precision", [1, 2])
def test_batch_fp32_close_to_per_level(mk, ctx, precision):
    ds = mixed_problems(precision)
    probs = [gpu_problem(mk, d, precision=precision) for d in ds]
    rb = ctx.estimate_batch(probs, mk.batch_config(pairs_per_thread=2, max_requests=64, max_nbins=128))
    for p, b in zip(probs, rb):
        r = ctx.estimate(p)
        nb = [lv["n"] for lv in b.levels]
        nr = [lv["n"] for lv in r.levels]
        assert all(abs(x - y) <= max(1, 1e-6 * y) for x, y in zip(nb, nr)), (nb, nr)
        if nb == nr:
            assert b.estimate == pytest.approx(r.estimate, rel=1e-6, abs=1e-9)
        if p.tol > 0:
            assert b.variance <= p.tol ** 2 / 2 * (1 + 1e-6)


def test_batch_deterministic_and_graph_equals_host_loop(mk, ctx):
    probs = [gpu_problem(mk, d, precision=1) for d in mixed_problems(1, seed=9)]
    g = mk.batch_config(pairs_per_thread=1, substeps_per_launch=64, use_graph=1, max_requests=64,
                        max_nbins=128)
    h = mk.batch_config(pairs_per_thread=1, substeps_per_launch=64, use_graph=0, max_requests=64,
                        max_nbins=128)
    a = ctx.estimate_batch(probs, g)
    b = ctx.estimate_batch(probs, g)
    c = ctx.estimate_batch(probs, h)
    for x, y, z in zip(a, b, c):
        assert x.estimate == y.estimate == z.estimate
        assert [lv["sy2"] for lv in x.levels] == [lv["sy2"] for lv in z.levels]


@pytest.mark.parametrize("ppt,slice_", [(1, 16), (2, 0), (4, 256), (8, 64)])
def test_batch_configs_agree(mk, ctx, ppt, slice_):
    """Kernel variants with other pairs-per-thread are separate compilations
    whose FP32 contractions may differ by an ulp per event: estimates agree to
    FP32 rounding, event counts exactly."""
    probs = [gpu_problem(mk, d, precision=2) for d in mixed_problems(2, seed=11)]
    ref = ctx.estimate_batch(probs, mk.batch_config(pairs_per_thread=1, substeps_per_launch=256,
                                                    max_requests=64, max_nbins=128))
    got = ctx.estimate_batch(probs, mk.batch_config(pairs_per_thread=ppt, substeps_per_launch=slice_,
                                                    max_requests=64, max_nbins=128))
    for x, y in zip(ref, got):
        if [lv["n"] for lv in x.levels] == [lv["n"] for lv in y.levels]:
            assert x.estimate == pytest.approx(y.estimate, rel=1e-6, abs=1e-9)
            for lx, ly in zip(x.levels, y.levels):
                assert lx["events_f"] == ly["events_f"]


def test_batch_estimates_meet_tolerance(mk, ctx):
    """E[x(T)^2] requests across eps: |estimate - closed form| within 4.5
    sigma of the reported statistical error (bias is zero for this QoI)."""
    ds = []
    for i, eps in enumerate((1.0, 0.3, 0.1, 0.03, 0.01)):
        ds.append(dict(eps=eps, T=0.5, dt0=0.1, M=2, L=3, qoi=0, init=0, nbins=0, tol=0.005,
                       n_warmup=100, seed=3, request=i))
    probs = [gpu_problem(mk, d, precision=1) for d in ds]
    for d, r in zip(ds, ctx.estimate_batch(probs, mk.batch_config(max_requests=64, max_nbins=128))):
        exact = W.msd_closed_form(d["eps"], d["T"])
        assert abs(r.estimate - exact) < 4.5 * math.sqrt(r.variance) + 1e-12
        assert r.variance <= d["tol"] ** 2 / 2 * (1 + 1e-6)


def test_batch_rejects_invalid(mk, ctx):
    cfg = mk.batch_config(max_requests=64, max_nbins=128)
    a = gpu_problem(mk, mixed_problems(1)[0], precision=1)
    b = gpu_problem(mk, mixed_problems(1)[2], precision=2)
    with pytest.raises(mk.MlkdError):
        ctx.estimate_batch([a, b], cfg)                      # mixed precision
    c = gpu_problem(mk, dict(mixed_problems(1)[2], seed=99), precision=1)
    with pytest.raises(mk.MlkdError):
        ctx.estimate_batch([a, c], cfg)                      # different seeds
    small = mk.batch_config(max_requests=64, max_nbins=8)
    d = gpu_problem(mk, mixed_problems(1)[1], precision=1)   # 32 bins
    with pytest.raises(mk.MlkdError):
        ctx.estimate_batch([d], small)


@pytest.mark.parametrize("refill_min", [1, 8])
def test_slice_length_changes_nothing(mk, ctx, refill_min):
    """A chunk stored at the end of a slice and resumed in the next (active
    and finished-but-unsummed lanes included) gives the same sums bit for
    bit, whatever the slice length."""
    probs = [gpu_problem(mk, d, precision=1) for d in mixed_problems(1, seed=17)]
    runs = [ctx.estimate_batch(probs, mk.batch_config(pairs_per_thread=2, substeps_per_launch=S,
                                                      max_requests=64, max_nbins=128,
                                                      refill_min=refill_min))
            for S in (0, 7, 64, 1000)]
    for rs in runs[1:]:
        for x, y in zip(runs[0], rs):
            assert x.estimate == y.estimate and x.variance == y.variance
            assert [lv["sy2"] for lv in x.levels] == [lv["sy2"] for lv in y.levels]
            if x.density is not None:
                assert np.array_equal(x.density, y.density)


def test_autotune_picks_from_grid(mk, ctx):
    probs = [gpu_problem(mk, d, precision=2) for d in mixed_problems(2, seed=13)[:3]]
    best, secs = ctx.autotune_batch(probs, mk.batch_config(max_requests=64, max_nbins=128))
    assert best.pairs_per_thread in (1, 2, 4, 8)
    assert best.substeps_per_launch in (16, 64, 256, 0)
    assert best.warp_pair_min_events in (0, -1, 4096)
    assert len(secs) == 48 and all(s > 0 for s in secs)
    assert min(secs) == pytest.approx(secs[[0, -1, 4096].index(best.warp_pair_min_events) * 16 +
                                          [1, 2, 4, 8].index(best.pairs_per_thread) * 4 +
                                          [16, 64, 256, 0].index(best.substeps_per_launch)])


def test_batch_with_level_sets(mk, ctx):
    """Requests over level sets in the batched form equal the per-level form."""
    ds = [dict(eps=0.1, T=1.0, dt0=0.5, M=2, L=6, qoi=1, init=1, nbins=0, tol=0.004,
               n_warmup=100, seed=5, request=10, level_set=[2, 4, 5, 6]),
          dict(eps=0.5, T=0.5, dt0=0.1, M=2, L=3, qoi=0, init=0, nbins=0, tol=0.01,
               n_warmup=100, seed=5, request=11, level_set=[0, 3])]
    probs = [gpu_problem(mk, d, precision=mk.PREC_FP64) for d in ds]
    rb = ctx.estimate_batch(probs, mk.batch_config(max_requests=64, max_nbins=128))
    for p, b in zip(probs, rb):
        r = ctx.estimate(p)
        assert [lv["n"] for lv in b.levels] == [lv["n"] for lv in r.levels]
        assert b.estimate == pytest.approx(r.estimate, rel=1e-12, abs=1e-14)


def test_refill_threshold_changes_only_sum_order(mk, ctx):
    """Restarting finished lanes one at a time or sixteen at a time runs the
    same pairs on the same streams: event counts equal, estimates equal to
    FP64 rounding of the sums (FP64 mode)."""
    probs = [gpu_problem(mk, d, precision=mk.PREC_FP64) for d in mixed_problems(0, seed=19)]
    cfg = dict(max_requests=64, max_nbins=128)
    fixed = [[lv["n"] for lv in r.levels] for r in ctx.estimate_batch(probs, mk.batch_config(**cfg))]
    probs = [gpu_problem(mk, dict(d, n_fixed=n, tol=0.0), precision=mk.PREC_FP64)
             for d, n in zip(mixed_problems(0, seed=19), fixed)]
    a = ctx.estimate_batch(probs, mk.batch_config(refill_min=1, **cfg))
    b = ctx.estimate_batch(probs, mk.batch_config(refill_min=16, **cfg))
    for x, y in zip(a, b):
        for lx, ly in zip(x.levels, y.levels):
            assert lx["n"] == ly["n"]
            assert lx["events_f"] == ly["events_f"] and lx["events_c"] == ly["events_c"]
            assert lx["sy2"] == pytest.approx(ly["sy2"], rel=1e-12)
        assert x.estimate == pytest.approx(y.estimate, rel=1e-12, abs=1e-15)
        if x.density is not None:
            np.testing.assert_allclose(x.density, y.density, rtol=1e-12, atol=1e-12)


def test_round_cut_by_chunk_capacity_continues(mk, ctx):
    """A level needing more pairs than one round holds (2048 chunks of at
    most eight times the target size: 2048 * 8 * 32 pairs at this level,
    where one pair per lane already fills a chunk) is split over several
    rounds with the same targets: pair and event counts equal those of the
    per-level form, which runs each level in one launch."""
    d = dict(eps=1e-3, T=1.0, dt0=0.5, M=2, L=9, qoi=1, init=1, nbins=0, seed=7, request=3,
             n_fixed=[1000] * 9 + [600_000])
    p = gpu_problem(mk, d, precision=mk.PREC_FP32_DY64)
    r = ctx.estimate(p)
    # one pair per lane, as the per-level form: sums agree to FP32 contraction
    (b,) = ctx.estimate_batch([p], mk.batch_config(max_requests=64, max_nbins=128,
                                                   warp_pair_min_events=-1))
    assert [lv["n"] for lv in b.levels] == d["n_fixed"] == [lv["n"] for lv in r.levels]
    for lb, lr in zip(b.levels, r.levels):
        assert lb["events_f"] == lr["events_f"] and lb["events_c"] == lr["events_c"]
        assert lb["sy"] == pytest.approx(lr["sy"], rel=1e-9, abs=1e-9)
    assert b.estimate == pytest.approx(r.estimate, rel=1e-9, abs=1e-12)
    # the deep level one pair per warp (the default): the same counts
    (w,) = ctx.estimate_batch([p], mk.batch_config(max_requests=64, max_nbins=128))
    assert [lv["n"] for lv in w.levels] == d["n_fixed"]
    for lw, lr in zip(w.levels, r.levels):
        assert abs(lw["events_f"] - lr["events_f"]) <= 1e-6 * lr["events_f"] + 2
        assert abs(lw["events_c"] - lr["events_c"]) <= 1e-6 * lr["events_c"] + 2


def test_full_size_periodic_step_matches_per_level_form(mk):
    """The benchmark's step at full size, in the configuration it times
    (one pair per lane, unbounded slices, CUDA graph, compensated FP32):
    N_l from the same adaptive pilot at tol 1e-3, then the three fixed-N
    estimates batched against the per-level form, whose pairs are pinned to
    the oracle one by one.  Pair counts equal; event counts, estimates and
    densities equal to FP32 rounding (separate compilations may round a
    flight's floor differently for a rare pair)."""
    cfg = mk.batch_config(pairs_per_thread=1, substeps_per_launch=0, use_graph=1, max_requests=16,
                          max_nbins=128, warp_pair_min_events=-1)
    ctx = mk.Context(0, arena_bytes=mk.batch_workspace_bytes(cfg))
    try:
        dicts = [dict(W.periodic_problem(e, seed=0, tol=1e-3), request=i)
                 for i, e in enumerate(W.PERIODIC_EPS)]
        prec = mk.PREC_FP32_COMP
        pilot = ctx.estimate_batch([mk.make_problem(precision=prec, **d) for d in dicts], cfg)
        fixed = [[lv["n"] for lv in r.levels] for r in pilot]
        assert sum(fixed[1]) > 2.5e7                       # the full size: about 9e6 level-0 pairs
        probs = [mk.make_problem(precision=prec, n_fixed=n, **d) for d, n in zip(dicts, fixed)]
        batched = ctx.estimate_batch(probs, cfg)
        for p, n, b in zip(probs, fixed, batched):
            r = ctx.estimate(p)
            assert [lv["n"] for lv in b.levels] == n == [lv["n"] for lv in r.levels]
            for lb, lr in zip(b.levels, r.levels):
                for k in ("events_f", "events_c"):
                    assert abs(lb[k] - lr[k]) <= 1e-6 * lr[k] + 2
            assert b.estimate == pytest.approx(r.estimate, rel=1e-6, abs=1e-9)
            np.testing.assert_allclose(b.density, r.density, rtol=0, atol=1e-3)
    finally:
        ctx.close()


def _exact_periodic(eps, dt, n):
    from oracle.kd_charfn import kd_charfn
    return 1.0 / 3.0 + kd_charfn(2 * math.pi, eps, dt, n) / (2 * math.pi ** 2)


@pytest.mark.parametrize("case", ["free_x2", "periodic"])
def test_mse_of_200_adaptive_estimates(mk, ctx, case):
    """Eq. mse (Sec. 4.1) over 200 independent adaptive estimates on the GPU.

    free_x2: E[x(T)^2] in free space, whose closed form
    2(T - eps^2 (1 - e^{-T/eps^2})) holds at every level, so the estimator is
    unbiased.  periodic: int x^2 f of the finest level's scheme, exact from the
    KD scheme's characteristic function.  With the standardised errors
    z_i = (estimate_i - exact)/sqrt(variance_i), the mean of z must be 0 within
    4.5 standard errors, and the mean of z^2 must lie between the 0.1 % and 99.9 %
    points of chi^2(200)/200.  Together these check the bias and the variance
    that the controller reports.  The MSE must also stay below the
    chi-square bound of tol^2/2."""
    from scipy import stats
    if case == "free_x2":
        base = dict(eps=0.5, T=0.5, dt0=0.1, M=2, L=3, qoi=0, init=0, nbins=0, tol=2e-3,
                    n_warmup=100)
        exact = W.msd_closed_form(0.5, 0.5)
    else:
        base = dict(eps=0.1, T=0.05, dt0=0.05, M=2, L=3, qoi=1, init=1, nbins=0, tol=2e-3,
                    n_warmup=100)
        exact = _exact_periodic(0.1, 0.05 / 8, 8)
    n_est = 200
    # One seed for a batch; the request ids separate the 200 streams.
    ds = [dict(base, seed=11, request=i) for i in range(n_est)]
    cfg = mk.batch_config(max_requests=64, max_nbins=128)
    res = []
    for k in range(0, n_est, 64):
        probs = [gpu_problem(mk, d, precision=mk.PREC_FP32_COMP) for d in ds[k:k + 64]]
        res += ctx.estimate_batch(probs, cfg)
    tol = base["tol"]
    est = np.array([r.estimate for r in res])
    var = np.array([r.variance for r in res])
    assert np.all(var <= tol * tol / 2 * (1 + 1e-9))
    z = (est - exact) / np.sqrt(var)
    assert abs(z.mean()) < 4.5 / math.sqrt(n_est), z.mean()
    lo, hi = stats.chi2.ppf([0.001, 0.999], n_est) / n_est
    assert lo < np.mean(z * z) < hi, np.mean(z * z)
    assert np.mean((est - exact) ** 2) < tol * tol / 2 * hi


@pytest.mark.parametrize("use_graph", [1, 0])
def test_publication_wait_runs_out_and_the_context_recovers(mk, ctx, use_graph):
    """The device's bounded wait for earlier queue reservations: with the test
    hook, every queue starts with places that are reserved and never
    published, so the first producer's wait (bounded at 1000 spins here) runs
    out.  The call must end with MLKD_ETIMEDOUT -- no fault, no hang, no
    unpublished place read -- and the context must serve the next call
    normally."""
    ds = mixed_problems(1, seed=13)[:3]
    probs = [gpu_problem(mk, d, precision=1) for d in ds]
    stall = mk.batch_config(pairs_per_thread=1, substeps_per_launch=256, use_graph=use_graph,
                            max_requests=64, max_nbins=128, publish_wait_spins=1000,
                            test_stall_queues=64)
    with pytest.raises(mk.MlkdError) as e:
        ctx.estimate_batch(probs, stall)
    assert e.value.status == mk.MLKD_ETIMEDOUT
    good = mk.batch_config(pairs_per_thread=1, substeps_per_launch=256, use_graph=use_graph,
                           max_requests=64, max_nbins=128)
    after = ctx.estimate_batch(probs, good)
    fresh = ctx.estimate_batch(probs, good)
    for a, b, d in zip(after, fresh, ds):
        assert a.estimate == b.estimate and a.variance == b.variance
        assert a.variance <= d["tol"] ** 2 / 2 * (1 + 1e-6)


WARP_PAIR_CASES = {
    # long diffusive chains (the deep levels of the periodic benchmark)
    "deep_diffusive": (dict(eps=1e-3, T=1.0, dt0=0.5, M=2, L=9, qoi=1, init=1, nbins=64, lo=0.0,
                            hi=1.0, seed=2, tol=0.0), 9, 300),
    # every regime through the warp path (threshold 1 event): kinetic,
    # mixed, drift, M = 3 and 8, free space with bins, single paths
    "kinetic": (dict(eps=2.0, T=1.0, dt0=0.25, M=2, L=3, qoi=0, init=0, nbins=0, seed=5, tol=0.0), 3, 2000),
    "mixed_periodic": (dict(eps=0.1, T=1.0, dt0=0.5, M=2, L=6, qoi=1, init=1, nbins=32, lo=0.0,
                            hi=1.0, seed=21, tol=0.0), 6, 2000),
    "M3_drift": (dict(eps=0.2, T=0.6, dt0=0.2, M=3, L=2, qoi=0, init=0, nbins=12, lo=-3.0, hi=3.0,
                      seed=17, mu=0.4, tol=0.0), 2, 2000),
    "M8": (dict(eps=0.05, T=1.0, dt0=0.5, M=8, L=2, qoi=0, init=0, nbins=0, seed=13, tol=0.0), 2, 2000),
    "single_paths": (dict(eps=0.05, T=1.0, dt0=0.5, M=2, L=3, qoi=0, init=0, nbins=0, seed=3, tol=0.0), 0, 2000),
}


@pytest.mark.parametrize("name", sorted(WARP_PAIR_CASES))
def test_warp_pair_form_matches_oracle_fp64(orc, mk, ctx, name):
    """Pairs run one per warp (32 events per step: step counts by prefix
    sum, coarse windows by their step index, window sums by segmented scan)
    give the oracle's pairs: the same fine and coarse event counts and
    positions within 1e-12 (the positions' FP sums are formed in another
    order).  The deep-diffusive case uses the default threshold (its pairs
    average more than 1024 events); the others force every level through
    the warp path."""
    d, level, n = WARP_PAIR_CASES[name]
    thr = 0 if name == "deep_diffusive" else 1
    nf = [n] * (d["L"] + 1)
    p = gpu_problem(mk, d, precision=mk.PREC_FP64, n_fixed=nf)
    cfg = mk.batch_config(pairs_per_thread=1, substeps_per_launch=0, max_requests=64, max_nbins=128,
                          warp_pair_min_events=thr)
    _, xf, xc, kf, kc = ctx.debug_batch_pairs(p, cfg, level)
    xf_o, xc_o, kf_o, kc_o = orc.pairs(oracle_problem(orc, d), level, 0, n, threads=16)
    assert np.array_equal(kf, kf_o) and np.array_equal(kc, kc_o)
    for g, o in ((xf, xf_o), (xc, xc_o)):
        assert np.all(np.abs(g - o) <= 1e-12 * np.maximum(1.0, np.abs(o))), np.max(np.abs(g - o))


def test_warp_pair_form_fp32_and_slices(orc, mk, ctx):
    """FP32 pairs of the warp path against the oracle on the 24-bit stream
    within the FP32 per-pair bound; and sliced launches (16 steps per
    launch, so pairs are stored and resumed mid-chain) equal the unsliced
    run bit for bit."""
    import fp32_bounds as B
    d, level, n = WARP_PAIR_CASES["deep_diffusive"]
    nf = [n] * (d["L"] + 1)
    p = gpu_problem(mk, d, precision=mk.PREC_FP32_COMP, n_fixed=nf)
    full = mk.batch_config(pairs_per_thread=1, substeps_per_launch=0, max_requests=64, max_nbins=128)
    r0, xf, xc, kf, kc = ctx.debug_batch_pairs(p, full, level)
    xf_o, xc_o, kf_o, kc_o = orc.pairs(oracle_problem(orc, d, recipe=orc.RECIPE_24), level, 0, n,
                                       threads=16)
    same = (kf == kf_o) & (kc == kc_o)
    assert (~same).sum() <= max(1, 1e-3 * n)
    ev = kf_o + kc_o
    for g, o in ((xf, xf_o), (xc, xc_o)):
        assert np.all(np.abs(g - o)[same] <= B.pair_delta(o, ev)[same])
    for ppt, sl in ((1, 16), (2, 64)):
        cfg = mk.batch_config(pairs_per_thread=ppt, substeps_per_launch=sl, max_requests=64,
                              max_nbins=128)
        r1, xf1, xc1, kf1, kc1 = ctx.debug_batch_pairs(p, cfg, level)
        if ppt == 1:
            assert np.array_equal(xf1, xf) and np.array_equal(xc1, xc)
            assert r1.estimate == r0.estimate
        assert np.array_equal(kf1, kf) and np.array_equal(kc1, kc)


LANE_POOL_CASES = {
    # R = 1/4 over T = 1: about 78 % of the pairs have no collision before T
    # and are finished in the start pass itself
    "kinetic_dead_starts": (dict(eps=2.0, T=1.0, dt0=0.25, M=2, L=3, qoi=0, init=0, nbins=16, lo=-3.0,
                                 hi=3.0, seed=8, tol=0.0), 2, 3001),
    "kinetic_single_paths": (dict(eps=2.0, T=1.0, dt0=0.25, M=2, L=3, qoi=0, init=0, nbins=16,
                                  lo=-3.0, hi=3.0, seed=8, tol=0.0), 0, 3001),
    "mixed_periodic": (dict(eps=0.1, T=1.0, dt0=0.5, M=2, L=6, qoi=1, init=1, nbins=32, lo=0.0,
                            hi=1.0, seed=21, tol=0.0), 4, 2001),
}


@pytest.mark.parametrize("name", sorted(LANE_POOL_CASES))
def test_lane_form_pools_match_oracle_fp64(orc, mk, ctx, name):
    """One pair per lane, with pairs started 32 at a time into a pool and
    finished pairs summed 32 at a time: every pair (those finished in the
    start pass included) is the oracle's pair, whatever the pairs per
    thread, the idle-lane threshold and the slice length.  The same
    configuration sliced or not gives the same sums bit for bit; another
    threshold or pairs-per-thread setting changes only their order."""
    d, level, n = LANE_POOL_CASES[name]
    nf = [n] * (d["L"] + 1)
    p = gpu_problem(mk, d, precision=mk.PREC_FP64, n_fixed=nf)
    xf_o, xc_o, kf_o, kc_o = orc.pairs(oracle_problem(orc, d), level, 0, n, threads=16)
    runs = {}
    for ppt, sl, rm in ((1, 0, 0), (1, 7, 0), (2, 0, 1), (2, 13, 1), (4, 5, 32), (1, 0, 3)):
        cfg = mk.batch_config(pairs_per_thread=ppt, substeps_per_launch=sl, max_requests=64,
                              max_nbins=128, refill_min=rm, warp_pair_min_events=-1)
        r, xf, xc, kf, kc = ctx.debug_batch_pairs(p, cfg, level)
        assert np.array_equal(kf, kf_o) and np.array_equal(kc, kc_o), (ppt, sl, rm)
        assert fp64_close(xf, xf_o).all() and fp64_close(xc, xc_o).all(), (ppt, sl, rm)
        runs[(ppt, sl, rm)] = r
    ref = runs[(1, 0, 0)]
    for key, r in runs.items():
        same_order = (key[0], key[2]) in ((1, 0), (2, 1)) and key[1] > 0
        base = ref if key[0] == 1 else runs[(2, 0, 1)]
        if same_order:
            assert r.estimate == base.estimate and r.variance == base.variance, key
        assert r.estimate == pytest.approx(ref.estimate, rel=1e-12, abs=1e-15), key
        for la, lb in zip(r.levels, ref.levels):
            assert la["events_f"] == lb["events_f"] and la["events_c"] == lb["events_c"]
