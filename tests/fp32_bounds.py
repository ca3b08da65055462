"""Error bounds of the FP32 modes' level sums and histograms (test helper).

The starting point is the per-pair bound of the FP32 pair state against the
oracle on the same 24-bit stream (tests/test_gpu_fp32.py): for a pair whose
event sequence equals the oracle's,

    |x_gpu - x_oracle| <= delta = C (events + 1) 2^-24 max(1, |x_oracle|).

Everything below propagates that bound through the quantity of interest of
eq. mlmc-compact (Sec. 4.1) and through the kernel's sums:

* F(x) = x^2: |F(x') - F(x)| <= (2|x| + delta) delta.
* F(x) = (x mod 1)^2: x mod 1 is exact in FP32 and F has slope 2 (x mod 1)
  <= 2, so |dF| <= (2 m + delta) delta with m = x mod 1, unless x lies within
  delta of an integer, where the wrap can move F anywhere in [0, 1).
* Y = F(x_f) - F(x_c): |dY| <= |dF_f| + |dF_c|; squares t^2 of a value t
  known to dt: |d(t^2)| <= (2|t| + dt) dt.
* FP32 formation of F, Y and their squares adds a few roundings of 2^-24 per
  term (a product, a difference, a possible multiply-add contraction).
* Summation: the compensated FP32 sums (TwoSum per addition, Sec. 4.1 sums in
  FP32_COMP; the F moments of FP32_DY64) have error at most
  u |S| + gamma_n^2 sum|t| (Ogita, Rump, Oishi 2005, Sum2), with u = 2^-24 and
  gamma_n = n u / (1 - n u); n is bounded by the pairs of the level.  FP64
  sums (Y and Y^2 of FP32_DY64, the rows and the oracle's numpy sum) add at
  most gamma_n(2^-53) sum|t|.

A histogram bin can differ only for pairs whose x lies within delta (plus the
FP32 rounding of the bin computation) of a bin edge; each such pair can move
one count between the two bins of that edge.
"""
import numpy as np

U32 = 2.0 ** -24
U64 = 2.0 ** -53
FP32_C = 16.0


def pair_delta(x, events, C=FP32_C):
    """Per-pair bound on |x_gpu - x_oracle| (events = fine + coarse)."""
    return C * (np.asarray(events, np.float64) + 1.0) * U32 * np.maximum(1.0, np.abs(x))


def qoi(periodic, x):
    """F(x) of the two scalar QoIs, in FP64."""
    if periodic:
        m = x - np.floor(x)
        return m * m
    return x * x


def qoi_change(periodic, x, d):
    """Bound on |F(x') - F(x)| over |x' - x| <= d, plus FP32 formation."""
    if periodic:
        m = x - np.floor(x)
        wrap = (m < d) | (m > 1.0 - d)
        # the slope bound, plus the FP32 rounding of x - floor(x) itself
        # (inexact only for small negative x, where the result is near 1)
        dF = np.where(wrap, 1.0, (2.0 * m + d) * d + 4.0 * U32 * m)
        F = m * m
    else:
        F = x * x
        dF = (2.0 * np.abs(x) + d) * d
    return dF + 2.0 * U32 * F


def square_change(t, dt, rounding):
    return (2.0 * np.abs(t) + dt) * dt + rounding * t * t


def gamma(n, u):
    nu = n * u
    return nu / (1.0 - nu)


def sum_error(terms, compensated, n):
    """Bound on the summation error of the kernel's sum of `terms`."""
    a = float(np.sum(np.abs(terms)))
    if compensated:
        return U32 * a + gamma(n, U32) ** 2 * a + gamma(n, U64) * a
    return gamma(n, U64) * a


def level_sum_bounds(periodic, coupled, xf, xc, ef, ec, precision):
    """For each of sy, sy2, sqf, sqf2, sqc, sqc2: the bound on
    |S_gpu - S_oracle| that the per-pair bound implies, given the oracle's
    pairs (positions, event counts) of one level.  precision: 1 = FP32_DY64
    (Y and Y^2 in FP64, F moments compensated FP32), 2 = FP32_COMP (all six
    compensated FP32)."""
    n = len(xf)
    ev = ef + ec
    df = pair_delta(xf, ev)
    Ff = qoi(periodic, xf)
    dFf = qoi_change(periodic, xf, df)
    if coupled:
        dc = pair_delta(xc, ev)
        Fc = qoi(periodic, xc)
        dFc = qoi_change(periodic, xc, dc)
    else:
        Fc = np.zeros(n)
        dFc = np.zeros(n)
    Y = Ff - Fc
    y_round = 4.0 * U32 * (Ff + Fc) if precision == 2 else 4.0 * U64 * (Ff + Fc)
    dY = dFf + dFc + y_round
    r_sq_y = 2.0 * U32 if precision == 2 else 2.0 * U64
    terms = {
        "sy": (Y, dY, precision == 2),
        "sy2": (Y * Y, square_change(Y, dY, r_sq_y), precision == 2),
        "sqf": (Ff, dFf, True),
        "sqf2": (Ff * Ff, square_change(Ff, dFf, 2.0 * U32), True),
        "sqc": (Fc, dFc, True),
        "sqc2": (Fc * Fc, square_change(Fc, dFc, 2.0 * U32), True),
    }
    out = {}
    for k, (t, dt, comp) in terms.items():
        # per-pair changes, the kernel's summation and the oracle's own sum
        out[k] = float(np.sum(dt)) + sum_error(t + dt, comp, n) + gamma(n, U64) * float(np.sum(np.abs(t)))
    return out


def edge_allowance(x, d, lo, hi, nbins, periodic):
    """Per-bin allowance of a histogram against the oracle: for each position
    whose distance to a bin edge is below d (plus FP32 rounding of the bin
    computation), one count for each of the two bins of that edge.  Returns
    (allowance[nbins], number of such positions)."""
    if periodic:
        x = x - np.floor(x)
    h = (hi - lo) / nbins
    t = (x - lo) / h                        # position in bin units
    k = np.rint(t)                          # nearest edge index
    dist = np.abs(t - k) * h
    slack = d * 1.001 + 8.0 * U32 * np.maximum(1.0, np.abs(x)) + 4.0 * U32 * h * nbins
    near = dist < slack
    allow = np.zeros(nbins, np.int64)
    ki = k[near].astype(np.int64)
    for side in (ki - 1, ki):               # the bins below and above the edge
        if periodic:
            side = np.mod(side, nbins)
        ok = (side >= 0) & (side < nbins)
        np.add.at(allow, side[ok], 1)
    return allow, int(np.count_nonzero(near))


def fp32_mod1(x64):
    """x - floor(x) of FP32 positions, rounded to FP32 as the kernel does."""
    x = np.asarray(x64, np.float64).astype(np.float32)
    return (x - np.floor(x)).astype(np.float32).astype(np.float64)


def fp32_bins(x64, lo, hi, nbins, periodic):
    """The kernel's FP32 bin decision for FP32 positions (exact replica:
    wrap x - floor(x), the range test, floor((x - lo) * (1/h)) and the top
    clamp, each rounded to FP32)."""
    x = np.asarray(x64, np.float64).astype(np.float32)
    lo_f, hi_f = np.float32(lo), np.float32(hi)
    inv_h = np.float32(1.0 / ((hi - lo) / nbins))
    if periodic:
        x = (x - np.floor(x)).astype(np.float32)
    inside = (x >= lo_f) & (x < hi_f)
    b = np.floor((x - lo_f).astype(np.float32) * inv_h).astype(np.int64)
    b = np.minimum(b, nbins - 1)
    return np.where(inside, b, -1)


def host_level_sums(periodic, coupled, xf, xc, precision):
    """The six sums of one level from FP32 positions (the kernel's own per-pair
    output), summed on the host in FP64, with a bound on how far the kernel's
    FP32 formation of each term can lie from this FP64 formation."""
    xf = np.asarray(xf, np.float64)
    xc = np.asarray(xc, np.float64) if coupled else np.zeros_like(xf)
    if periodic:
        # x mod 1 exactly as the kernel forms it: x - floor(x) rounded to FP32
        mf = fp32_mod1(xf)
        mc = fp32_mod1(xc) if coupled else np.zeros_like(mf)
        Ff, Fc = mf * mf, mc * mc
        Y = Ff - Fc
    else:
        Ff, Fc = xf * xf, xc * xc
        Y = Ff - Fc if not coupled else (xf - xc) * (xf + xc)
    if not coupled:
        Fc = np.zeros_like(Ff)
    rf = 4.0 * U32 * np.maximum(1.0, Ff)       # F formed in FP32
    rc = 4.0 * U32 * np.maximum(1.0, Fc) if coupled else np.zeros_like(Fc)
    ry = (rf + rc + 4.0 * U32 * np.abs(Y)) if precision == 2 else 4.0 * U64 * (Ff + Fc + np.abs(Y))
    sums = {"sy": Y, "sy2": Y * Y, "sqf": Ff, "sqf2": Ff * Ff, "sqc": Fc, "sqc2": Fc * Fc}
    form = {"sy": ry, "sy2": square_change(Y, ry, 2.0 * (U32 if precision == 2 else U64)),
            "sqf": rf, "sqf2": square_change(Ff, rf, 2.0 * U32),
            "sqc": rc, "sqc2": square_change(Fc, rc, 2.0 * U32)}
    return ({k: float(np.sum(v)) for k, v in sums.items()},
            {k: float(np.sum(v)) for k, v in form.items()},
            {k: v for k, v in sums.items()})
