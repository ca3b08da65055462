"""KD coefficients of eqs. advection/diffusion and the aggregation quantities of
Sec. 3.2 as the pair kernels compute them (mlkd_debug_kd_coeffs), against the
oracle's FP64 formulas (GPU only).

FP64 state: the same closed forms and series, so the values agree to FP64
rounding.  FP32 state: compared with the oracle evaluated at the FP32-rounded
inputs, within bounds derived from the arithmetic:

* the series branch (s = R theta < 1) evaluates h, f, g as Chebyshev
  interpolants with at most 2.7 ulp error, then a few products;
* the exponential branch (s >= 1) forms f = 2(e - 1) + s(e + 1) and
  g = 1 - 2 s e - e^2 with e = exp(-s): their rounding errors scale with the
  terms, not with f or g, so the bound is taken on the sum of |terms|;
* s itself is rounded once (R theta in FP32).

Each bound is K u times the size of the terms that form the quantity (u =
2^-24 for FP32, 2^-53 for FP64); the tests print the largest error in units
of its bound.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24

# diffusive scaling R = 1/eps^2, sigma = 1/eps, and one drifting background
BACKGROUNDS = [(4.0, 0.0, 2.0), (100.0, 0.0, 10.0), (1.0e4, 0.3, 100.0), (1.0e6, 0.0, 1000.0)]


@pytest.fixture(scope="module")
def mk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_04071_gb300 as mk
    mk.lib()
    return mk


def inputs(R, sigma, n, seed):
    rng = np.random.default_rng(seed)
    s = np.concatenate([10.0 ** rng.uniform(-5.0, 2.5, n - 9),
                        [0.5, 0.999, 0.9999999, 1.0, 1.0000001, 1.001, 2.0, 30.0, 200.0]])
    theta = s / R
    dv = sigma * rng.standard_normal(theta.size)
    return theta, dv


def oracle_values(orc, R, mu, sigma, theta, dv):
    L = orc.lib()
    a = np.array([L.orc_advection(R, mu, t, mu + w) for t, w in zip(theta, dv)])
    d = np.array([L.orc_diffusion(R, mu, sigma, t, mu + w) for t, w in zip(theta, dv)])
    s = R * theta
    hs = np.array([L.orc_hs(x) for x in s])
    om = -np.expm1(-s)
    bh2 = np.array([2.0 * L.orc_hs(h) for h in hs])
    return a, d, hs, om, bh2


def gpu_values(mk, precision, R, mu, sigma, theta, dv):
    import torch
    t = torch.tensor(theta, dtype=torch.float64, device="cuda:0")
    w = torch.tensor(dv, dtype=torch.float64, device="cuda:0")
    return [x.cpu().numpy() for x in mk.debug_kd_coeffs(precision, R, mu, sigma, t, w)]


def bounds(R, mu, sigma, theta, dv, hs, om, d, u, K, s_kernel):
    """Absolute error bounds of (a, d, hs, om, bh2): K u times the sizes of
    the terms that form each quantity.  The branch (series or exponential)
    is the one the kernel took, decided on its own s."""
    s = R * theta
    e = np.exp(-s)
    big = s_kernel >= 1.0
    # rounding errors scale with the terms, not with the result (the
    # exponential branch cancels)
    f_terms = np.where(big, 2.0 * np.abs(e - 1.0) + s * (e + 1.0), s ** 3 / 6.0)
    g_terms = np.where(big, 1.0 + 2.0 * s * e + e * e, 2.0 * s ** 3 / 3.0)
    h_terms = np.where(big, s + 1.0 + e, s * s / 2.0)
    hh_terms = np.where(hs >= 1.0, hs + 1.0 + np.exp(-hs), hs * hs / 2.0)
    d2_terms = 2.0 * sigma ** 2 / R ** 2 * f_terms + (dv / R) ** 2 * g_terms
    a_terms = np.abs(mu * theta) + np.abs(dv) * om / R
    return {
        "a": K * u * a_terms,
        # d = sqrt(d^2): an error of d^2 moves d by that error / 2d, plus the root's own
        "d": K * u * d2_terms / (2.0 * np.maximum(d, 1e-300)) + 2.0 * u * d,
        "hs": K * u * h_terms,
        "om": K * u * om,
        # 2 h(hs): its own evaluation, plus the error of hs through h'(hs) = 1 - e^{-hs}
        "bh2": 2.0 * K * u * hh_terms + 2.0 * np.minimum(hs, 1.0) * K * u * h_terms,
    }


def check(name_vals, bnd, label):
    for name, g, o in name_vals:
        ratio = np.abs(g - o) / np.maximum(bnd[name], 1e-300)
        worst = float(np.max(ratio))
        print("%s %s: worst error %.3f of its bound" % (label, name, worst))
        assert worst <= 1.0, (label, name, worst)


@pytest.mark.parametrize("R,mu,sigma", BACKGROUNDS)
def test_fp64_coefficients_equal_the_oracle(orc, mk, R, mu, sigma):
    """The FP64 kernel evaluates the same formulas as the oracle (its series
    have more terms than FP64 needs): both agree to a few FP64 roundings of
    the terms (K = 16, u = 2^-53)."""
    theta, dv = inputs(R, sigma, 4000, 1)
    a, d, hs, om, bh2 = oracle_values(orc, R, mu, sigma, theta, dv)
    got = gpu_values(mk, mk.PREC_FP64, R, mu, sigma, theta, dv)
    bnd = bounds(R, mu, sigma, theta, dv, hs, om, d, 2.0 ** -53, 16.0, R * theta)
    check(zip(("a", "d", "hs", "om", "bh2"), got, (a, d, hs, om, bh2)), bnd, "FP64 R=%g" % R)


@pytest.mark.parametrize("R,mu,sigma", BACKGROUNDS)
def test_fp32_coefficients_within_derived_bounds(orc, mk, R, mu, sigma):
    """FP32 state against the oracle at the FP32-rounded inputs, K = 8,
    u = 2^-24."""
    theta, dv = inputs(R, sigma, 20000, 2)
    theta32 = theta.astype(np.float32).astype(np.float64)
    dv32 = dv.astype(np.float32).astype(np.float64)
    a, d, hs, om, bh2 = oracle_values(orc, R, mu, sigma, theta32, dv32)
    got = gpu_values(mk, mk.PREC_FP32_COMP, R, mu, sigma, theta, dv)
    s32 = (np.float32(R) * theta32.astype(np.float32)).astype(np.float64)
    bnd = bounds(R, mu, sigma, theta32, dv32, hs, om, d, U32, 8.0, s32)
    check(zip(("a", "d", "hs", "om", "bh2"), got, (a, d, hs, om, bh2)), bnd, "FP32 R=%g" % R)
