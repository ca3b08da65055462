"""Seeded synthetic workloads of the correlated-pair path.

Plain parameter sets and seeded request streams, shared by the tests, the
benchmark and the CPU baseline.  Nothing here computes any part of the
method: the Monte Carlo random numbers are drawn inside the oracle and inside
the CUDA library from their own Philox streams.

The paper measures on analytic backgrounds, not on a dataset; these are the
free-space and periodic homogeneous problems in the diffusive scaling
(R = 1/eps^2, sigma = 1/eps, mu = 0).
"""
from __future__ import annotations

import math

import numpy as np

QOI_X2, QOI_X2_PERIODIC, QOI_DENSITY = 0, 1, 2
INIT_ORIGIN, INIT_COSINE = 0, 1


def msd_closed_form(eps: float, T: float) -> float:
    """E[x(T)^2] of the kinetic process from x = 0 with unit-variance velocities
    in the diffusive scaling: 2 (T - eps^2 (1 - exp(-T/eps^2)))."""
    return 2.0 * (T - eps * eps * (1.0 - math.exp(-T / (eps * eps))))


# Two-level free-space problem: x0 = 0, eps = 0.5, T = 0.5, dt0 = 0.1, M = 2,
# N_0 = 10^4 single paths and N_1 = 2000 pairs; QoI E[x^2] plus 20 bins on [-3, 3).
TWO_LEVEL = dict(eps=0.5, T=0.5, dt0=0.1, M=2, L=1, qoi=QOI_X2, init=INIT_ORIGIN, nbins=20,
                 lo=-3.0, hi=3.0, seed=0, n_fixed=[10_000, 2_000])


def periodic_levels(eps: float, dt0: float = 0.5, cap: int = 12) -> int:
    """Finest level of the periodic problem: dt_L <= eps^2/4, at most `cap`."""
    return min(cap, max(1, math.ceil(math.log2(dt0 / (eps * eps / 4.0)))))


# Full periodic MLMC: density 1 + cos(2 pi x) on [0, 1), T = 1, dt0 = 0.5,
# M = 2, eps in {1, 0.1, 1e-3}, RMSE tolerance 1e-3; QoI int x^2 f and 128 bins.
PERIODIC_EPS = (1.0, 0.1, 1e-3)


def periodic_problem(eps: float, seed: int = 0, tol: float = 1e-3) -> dict:
    return dict(eps=eps, T=1.0, dt0=0.5, M=2, L=periodic_levels(eps), qoi=QOI_X2_PERIODIC,
                init=INIT_COSINE, nbins=128, lo=0.0, hi=1.0, tol=tol, n_warmup=100, seed=seed)


# Precision study: the two-level free-space geometry at eps = 1e-2, tol = 1e-4.
def precision_problem(seed: int = 0) -> dict:
    return dict(eps=1e-2, T=0.5, dt0=0.1, M=2, L=1, qoi=QOI_X2, init=INIT_ORIGIN, nbins=0,
                tol=1e-4, n_warmup=100, seed=seed)


def batched_requests(n: int = 64, seed: int = 0) -> list:
    """64 independent estimators: eps log-uniform in [1e-4, 1], tol log-uniform
    in [1e-4, 1e-2], L = clamp(ceil(log2(4 dt0/eps^2)), 2, 13); even requests
    estimate E[x^2] from x = 0 (T = 0.5, dt0 = 0.1), odd ones the periodic
    int x^2 f from the cosine start (T = 1, dt0 = 0.5)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        eps = float(10.0 ** rng.uniform(-4.0, 0.0))
        tol = float(10.0 ** rng.uniform(-4.0, -2.0))
        if i % 2 == 0:
            T, dt0, qoi, init, nb = 0.5, 0.1, QOI_X2, INIT_ORIGIN, 0
        else:
            T, dt0, qoi, init, nb = 1.0, 0.5, QOI_X2_PERIODIC, INIT_COSINE, 0
        L = int(min(13, max(2, math.ceil(math.log2(4.0 * dt0 / (eps * eps))))))
        out.append(dict(eps=eps, T=T, dt0=dt0, M=2, L=L, qoi=qoi, init=init, nbins=nb,
                        lo=0.0, hi=1.0, tol=tol, n_warmup=100, seed=seed, request=i))
    return out


def serving_stream(n: int = 2000, rate: float = 200.0, seed: int = 0) -> list:
    """Poisson arrivals at `rate` req/s; eps log-uniform in [1e-4, 1], tol
    log-uniform in [1e-4, 5e-3]; QoI E[x^2] from x = 0 or a 64-bin density
    from the cosine start, half each."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate))
        eps = float(10.0 ** rng.uniform(-4.0, 0.0))
        tol = float(10.0 ** rng.uniform(math.log10(1e-4), math.log10(5e-3)))
        if rng.random() < 0.5:
            T, dt0, qoi, init, nb = 0.5, 0.1, QOI_X2, INIT_ORIGIN, 0
        else:
            T, dt0, qoi, init, nb = 1.0, 0.5, QOI_DENSITY, INIT_COSINE, 64
        L = int(min(13, max(2, math.ceil(math.log2(4.0 * dt0 / (eps * eps))))))
        out.append(dict(arrival=t, eps=eps, T=T, dt0=dt0, M=2, L=L, qoi=qoi, init=init,
                        nbins=nb, lo=0.0, hi=1.0, tol=tol, n_warmup=100, seed=seed, request=i))
    return out
