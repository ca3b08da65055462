"""The FP32 variate transforms of the pair kernel, checked exhaustively over
all 2^24 uniforms u = n 2^-24 against double-precision references (GPU
only): log u by the atanh series, sin/cos of 2 pi u by quarter-turn reduction
and Taylor polynomials."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_log_sin_cos_of_all_24_bit_uniforms():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_04071_gb300 as mk
    n = np.arange(1 << 24, dtype=np.int64)                 # word w = n << 8 -> u = (n + 1) 2^-24
    words = torch.tensor((n << 8).astype(np.uint32).view(np.int32), device="cuda")
    lg = torch.empty(1 << 24, dtype=torch.float32, device="cuda")
    sn = torch.empty_like(lg)
    cs = torch.empty_like(lg)
    mk.debug_transforms(words, lg, sn, cs)
    lg, sn, cs = (t.cpu().numpy().astype(np.float64) for t in (lg, sn, cs))
    u = (n + 1).astype(np.float64) * 2.0 ** -24
    ref_log = np.log(u)
    ulp = np.spacing(np.abs(ref_log).astype(np.float32)).astype(np.float64)
    err_log = np.abs(lg - ref_log)
    # a few ulp of the result
    assert np.all(err_log <= 4 * np.maximum(ulp, 2.0 ** -149))
    assert lg[-1] == 0.0
    ref_s, ref_c = np.sin(2 * np.pi * u), np.cos(2 * np.pi * u)
    assert np.max(np.abs(sn - ref_s)) <= 2.0 ** -22
    assert np.max(np.abs(cs - ref_c)) <= 2.0 ** -22
    assert np.max(np.abs(sn * sn + cs * cs - 1.0)) <= 2.0 ** -21
