"""The debug build with device checks (libmlkd_checked.so; GPU only).

A subprocess loads the checked library (MLKD_CHECKED=1) and runs the forms of
the path on small cases: per-level launches with histograms, the adaptive
per-level estimate, the batched form sliced, with one pair per warp and with
the heterogeneous backgrounds, and the per-pair readouts.  No check may fail,
and the results must equal the normal library's.  The self-test launches a
kernel whose check fails on purpose: the failure is recorded (no access out
of bounds, no trap) and reported as MLKD_EINTERNAL.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from helpers import gpu_problem

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = {
    "periodic": dict(eps=0.1, T=1.0, dt0=0.5, M=2, L=5, qoi=2, init=1, nbins=32, lo=0.0, hi=1.0,
                     seed=3),
    "free": dict(eps=0.5, T=0.5, dt0=0.1, M=2, L=3, qoi=0, init=0, nbins=20, lo=-3.0, hi=3.0, seed=1),
    "hetero": dict(eps=1.0, T=1.0, dt0=0.5, M=2, L=4, qoi=3, init=2, x0=1.0, nbins=16, lo=-1.0,
                   hi=3.0, seed=0, background=1, bg_a=10.0, bg_b=100.0),
}

SCRIPT = r"""
import json, sys
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import paper_2004_04071_gb300 as mk
from helpers import gpu_problem
import test_gpu_checked as T
print(json.dumps(T.run_all(mk, gpu_problem)))
"""


def run_all(mk, gpu_problem):
    """The checked calls; returns the results and the check state."""
    out = {"checks": list(mk.device_checks())}
    ctx = mk.Context(0, arena_bytes=mk.batch_workspace_bytes(mk.batch_config(max_requests=64,
                                                                              max_nbins=128)))
    for name, d in CASES.items():
        p = gpu_problem(mk, d, precision=mk.PREC_FP64)
        lv = ctx.run_level(p, 2, 0, 3000)
        out[name + "_level"] = [float(lv["sy"]), float(lv["sy2"]), int(lv["events_f"]),
                                int(lv["events_c"]), [int(x) for x in lv["hist_f"]]]
        xf, xc, kf, kc = ctx.debug_pairs(p, 1, 0, 500)
        out[name + "_pairs"] = [float(np.sum(xf)), float(np.sum(xc)), int(np.sum(kf)), int(np.sum(kc))]
        r = ctx.estimate(gpu_problem(mk, dict(d, tol=0.02), precision=mk.PREC_FP64))
        out[name + "_estimate"] = [float(r.estimate), [int(x["n"]) for x in r.levels]]
        nf = [600] * (d["L"] + 1)
        pf = gpu_problem(mk, dict(d, n_fixed=nf), precision=mk.PREC_FP64)
        for sl, wp in ((0, 0), (7, 1), (64, -1)):
            cfg = mk.batch_config(pairs_per_thread=2, substeps_per_launch=sl, max_requests=64,
                                  max_nbins=128, warp_pair_min_events=wp)
            rb, bxf, bxc, bkf, bkc = ctx.debug_batch_pairs(pf, cfg, 1)
            out["%s_batch_%d_%d" % (name, sl, wp)] = [float(rb.estimate), float(np.sum(bxf)),
                                                       int(np.sum(bkf))]
    out["after_runs"] = list(mk.device_checks())
    out["selftest"] = mk.debug_check_selftest(0)
    out["after_selftest"] = list(mk.device_checks())
    if mk.device_checks()[0]:
        # A stray write, made on the host: the first canary of the arena sits
        # right after the 16 level slots of block partial rows (16 x 4096 x 8
        # doubles); the next call must report it.
        ctx.arena[16 * 4096 * 8 * 8] = 0
        try:
            ctx.run_level(gpu_problem(mk, CASES["free"], precision=mk.PREC_FP64), 1, 0, 100)
            out["after_corruption"] = mk.MLKD_OK
        except mk.MlkdError as e:
            out["after_corruption"] = e.status
    ctx.close()
    return out


@pytest.fixture(scope="module")
def checked():
    pytest.importorskip("torch")
    env = dict(os.environ, MLKD_CHECKED="1")
    script = SCRIPT.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, env=env,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_is_loaded_and_clean(checked):
    assert checked["checks"] == [1, 0]
    assert checked["after_runs"] == [1, 0]


def test_selftest_reports_a_failed_check(checked):
    import paper_2004_04071_gb300 as mk
    assert checked["selftest"] == mk.MLKD_EINTERNAL
    assert checked["after_selftest"][0] == 1 and checked["after_selftest"][1] > 0


def test_canary_reports_a_stray_write(checked):
    """The debug build surrounds the arena regions with canary bytes and
    compares them after each synchronising call: a byte changed behind the
    library's back gives MLKD_EINTERNAL."""
    import paper_2004_04071_gb300 as mk
    assert checked["after_corruption"] == mk.MLKD_EINTERNAL


def _same(a, b):
    """Equal structure: floats to 1e-13 relative, everything else exactly."""
    if isinstance(a, list):
        return isinstance(b, list) and len(a) == len(b) and all(_same(x, y) for x, y in zip(a, b))
    if isinstance(a, float) or isinstance(b, float):
        return bool(np.isclose(a, b, rtol=1e-13, atol=1e-15))
    return a == b


def test_checked_results_equal_the_normal_build(checked):
    """The checks change no arithmetic: the normal library gives the same
    results (FP64, to 1e-13)."""
    import paper_2004_04071_gb300 as mk
    assert mk.device_checks()[0] == 0
    normal = json.loads(json.dumps(run_all(mk, gpu_problem)))
    assert normal["selftest"] == mk.MLKD_ENOTFOUND
    for key, val in checked.items():
        if key in ("checks", "after_runs", "selftest", "after_selftest", "after_corruption"):
            continue
        assert _same(val, normal[key]), (key, val, normal[key])
