"""Shared test helpers: one problem dict -> oracle Problem and C-ABI Problem."""
import numpy as np

ORACLE_KEYS = ("eps", "T", "dt0", "M", "L", "qoi", "init", "nbins", "lo", "hi", "tol",
               "n_warmup", "seed", "request", "mu", "x0")
BG_KEYS = ("background", "bg_a", "bg_b")


def oracle_problem(orc, d, recipe=None, **over):
    d = dict(d, **over)
    kw = {k: d[k] for k in ORACLE_KEYS if k in d}
    if d.get("background"):
        kw["background"], kw["a"], kw["b"] = d["background"], d.get("bg_a", 0.0), d["bg_b"]
    if "n_fixed" in d and d["n_fixed"] is not None:
        kw["n_fixed"] = list(d["n_fixed"])
    if recipe is not None:
        kw["recipe"] = recipe
    if d.get("level_set"):
        kw["level_set"] = list(d["level_set"])
    return orc.Problem(**kw)


def gpu_problem(mk, d, precision=0, **over):
    d = dict(d, **over)
    kw = {k: d[k] for k in ORACLE_KEYS + BG_KEYS if k in d}
    if "n_fixed" in d:
        kw["n_fixed"] = d["n_fixed"]
    if d.get("level_set"):
        kw["level_set"] = d["level_set"]
    return mk.make_problem(precision=precision, **kw)


def fp64_close(a, b, rel=1e-12):
    """|a - b| <= rel * max(1, |b|), elementwise."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) <= rel * np.maximum(1.0, np.abs(b))


def level_curve(level_sums, L, n):
    """(dt_l, V_{l,l-1}, C_{l,l-1}) for l = 1..L of the free-space x^2 QoI from
    level sums returned by `level_sums(level, n)` as (sy, sy2, n, events)."""
    out = []
    for l in range(1, L + 1):
        sy, sy2, cnt, ev = level_sums(l, n)
        out.append((0.5 / 2 ** l, (sy2 - sy * sy / cnt) / (cnt - 1), ev / cnt))
    return out


def check_level_curve(curve, R):
    """Sec. 5.2: maximum of V_{l,l-1} within a factor 2 of dt = 1/R; below
    dt = 1/(8R) each halving divides it by about 8 (dt^3); above the maximum
    each halving multiplies the cost per pair by about 2 and below dt = 1/(8R)
    leaves it flat."""
    dts = np.array([c[0] for c in curve])
    V = np.array([c[1] for c in curve])
    C = np.array([c[2] for c in curve])
    k = int(np.argmax(V))
    assert 0.5 / R <= dts[k] <= 2.0 / R, (dts[k], 1.0 / R)
    small = np.nonzero(dts <= 1.0 / (8 * R))[0]
    assert small.size >= 3
    ratios = V[small[:-1]] / V[small[1:]]
    assert np.all((ratios > 5.0) & (ratios < 12.0)), ratios
    big = np.nonzero(dts >= 8.0 / R)[0]
    cr = C[big[1:]] / C[big[:-1]]
    assert big.size >= 2 and np.all((cr > 1.6) & (cr < 2.4)), cr
    flat = C[small[1:]] / C[small[:-1]]
    assert np.all((flat > 0.9) & (flat < 1.15)), flat
