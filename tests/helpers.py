"""Shared test helpers: one problem dict -> oracle Problem and C-ABI Problem."""
import numpy as np

ORACLE_KEYS = ("eps", "T", "dt0", "M", "L", "qoi", "init", "nbins", "lo", "hi", "tol",
               "n_warmup", "seed", "request", "mu")


def oracle_problem(orc, d, recipe=None, **over):
    d = dict(d, **over)
    kw = {k: d[k] for k in ORACLE_KEYS if k in d}
    if "n_fixed" in d and d["n_fixed"] is not None:
        kw["n_fixed"] = list(d["n_fixed"])
    if recipe is not None:
        kw["recipe"] = recipe
    if d.get("level_set"):
        kw["level_set"] = list(d["level_set"])
    return orc.Problem(**kw)


def gpu_problem(mk, d, precision=0, **over):
    d = dict(d, **over)
    kw = {k: d[k] for k in ORACLE_KEYS if k in d}
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
