"""The allocation-free entry point (GPU only).

mlkd_run_level_noalloc exists for callers that may not allocate device
memory at all (an application allocator that must own every device byte, a
plugin host that forbids cudaMalloc).  Its scratch is a static device array
shared by every call.  This test calls it through the C ABI several times in
a row -- with and without a histogram, so stale counters from an earlier call
would show -- checks each result against mlkd_run_level on a context, and
checks that the calls leave the device's free memory unchanged.
It lives in its own file, collected after every other test.
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from helpers import gpu_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_04071_gb300 as mk
    mk.lib()
    return mk


def _noalloc(mk, problem, level, first, n):
    import torch
    st = mk.LevelStats()
    hist = np.zeros(max(1, 3 * problem.nbins), np.uint64)
    hp = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)) if problem.nbins else None
    rc = mk.lib().mlkd_run_level_noalloc(ctypes.byref(problem), level, first, n,
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                         ctypes.byref(st), hp)
    return rc, st.as_dict(), hist[:3 * problem.nbins]


def _close(a, b, rel=1e-12):
    return abs(a - b) <= rel * max(1.0, abs(b))


def _check_same(mk, p, got, hist, ref, n):
    assert got["n"] == ref["n"] == n
    assert got["events_f"] == ref["events_f"] and got["events_c"] == ref["events_c"]
    for key in ("sy", "sy2", "sqf", "sqf2", "sqc", "sqc2"):
        assert _close(got[key], ref[key]), (key, got[key], ref[key])
    if p.nbins:
        nb = p.nbins
        assert np.array_equal(hist[:nb], ref["hist_f"])
        assert np.array_equal(hist[nb:2 * nb], ref["hist_c"])
        assert np.array_equal(hist[2 * nb:], ref["hist_both"])


def test_noalloc_matches_run_level_on_consecutive_calls(mk):
    """Each case is called twice in a row, after every kernel variant it uses
    has been loaded once.  Between the first and the last of those calls the
    device's free memory and torch's allocator counters must not move: the
    entry point allocates nothing."""
    import torch
    ctx = mk.Context(0)
    try:
        cases = [
            (dict(W.TWO_LEVEL, n_fixed=None), 1, 0, 30000, mk.PREC_FP64),
            (W.periodic_problem(0.1), 3, 5, 20000, mk.PREC_FP32_DY64),
            (dict(eps=0.5, T=0.5, dt0=0.1, M=2, L=2, seed=7), 2, 100, 10000, mk.PREC_FP32_COMP),
            (dict(W.TWO_LEVEL, n_fixed=None), 1, 0, 30000, mk.PREC_FP64),
        ]
        probs = [(gpu_problem(mk, d, precision=prec), level, first, n)
                 for d, level, first, n, prec in cases]
        refs = [ctx.run_level(p, level, first, n) for p, level, first, n in probs]
        for p, level, first, n in probs:          # loads every kernel variant once
            rc, _, _ = _noalloc(mk, p, level, first, n)
            assert rc == mk.MLKD_OK, mk.status_string(rc)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(0)[0]
        alloc0, reserved0 = torch.cuda.memory_allocated(0), torch.cuda.memory_reserved(0)
        for (p, level, first, n), ref in zip(probs, refs):
            for _ in range(2):
                rc, got, hist = _noalloc(mk, p, level, first, n)
                assert rc == mk.MLKD_OK, mk.status_string(rc)
                _check_same(mk, p, got, hist, ref, n)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info(0)[0] == free0
        assert torch.cuda.memory_allocated(0) == alloc0
        assert torch.cuda.memory_reserved(0) == reserved0
    finally:
        ctx.close()


def test_noalloc_rejects_too_many_bins(mk):
    d = W.periodic_problem(0.1)
    p = gpu_problem(mk, d, nbins=mk.NOALLOC_MAX_BINS + 1)
    rc, _, _ = _noalloc(mk, p, 1, 0, 1000)
    assert rc == mk.MLKD_ENOMEM
