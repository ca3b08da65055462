"""Checkpoint and resume of an adaptive estimate (GPU only): a run stopped
after some rounds (a controller that dies mid-estimate) and restarted from
its saved level sums, pair counts and histogram counts ends exactly as the
uninterrupted run, also through the text form of the checkpoint."""
import numpy as np
import pytest

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


CASES = [
    (dict(eps=0.5, T=0.5, dt0=0.1, M=2, L=3, qoi=0, init=0, nbins=20, lo=-3.0, hi=3.0, tol=0.004,
          n_warmup=100, seed=4), 0),
    # periodic x^2 with a 16-bin density on the side: three rounds after the
    # warm-up (the oracle on the same 24-bit stream takes three)
    (dict(eps=0.2, T=1.0, dt0=0.5, M=2, L=4, qoi=1, init=1, nbins=16, lo=0.0, hi=1.0, tol=0.004,
          n_warmup=100, seed=6), 1),
]


@pytest.mark.parametrize("d,precision", CASES)
def test_resume_equals_uninterrupted(mk, d, precision):
    ctx = mk.Context(0)
    try:
        p = gpu_problem(mk, d, precision=precision)
        full, hfull = ctx.estimate_resumable(p)
        assert full.rounds >= 2, "the case must need several rounds"
        part, hpart = ctx.estimate_resumable(p, max_rounds=1)
        assert part.rounds == 1
        text = mk.checkpoint_to_json(part, hpart)
        ck, hck = mk.checkpoint_from_json(text)
        rest, hrest = ctx.estimate_resumable(p, resume=ck, hist_in=hck)
        assert rest.rounds == full.rounds
        assert rest.estimate == full.estimate and rest.variance == full.variance
        assert rest.levels == full.levels
        assert np.array_equal(rest.density, full.density)
        assert np.array_equal(hrest, hfull)
        # and the resumable call without a limit is mlkd_estimate itself
        plain = ctx.estimate(p)
        assert plain.estimate == full.estimate and plain.levels == full.levels
    finally:
        ctx.close()
