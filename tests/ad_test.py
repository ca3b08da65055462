"""Anderson-Darling test of a sample against a fully specified law (test
helper), as used in the consistency check of Sec. 5.1 (eq. anderson).

A^2 = -N - sum_i (2i - 1)/N [ln F(x_(i)) + ln(1 - F(x_(N+1-i)))] for the
sorted sample.  Its p-value comes from the limiting distribution of A^2 for a
fully specified law (Anderson and Darling, 1954):

  P(A^2 <= z) = sqrt(2 pi)/z sum_{j>=0} binom(-1/2, j) (4j+1)
                e^{-(4j+1)^2 pi^2/(8z)}
                int_0^inf exp(z/(8(w^2+1)) - (4j+1)^2 pi^2 w^2/(8z)) dw,

summed here with numerical quadrature.  tests/golden/ad_table_hypothesis.txt
holds (A^2, p) pairs printed in the paper's Table hypothesis, which this
reproduces to the printed digits (test_oracle_statistics.py).
"""
import math

import numpy as np
from scipy import integrate


def ad_statistic(x, cdf):
    """A^2 of sample x against the CDF `cdf` (vectorised callable)."""
    x = np.sort(np.asarray(x, np.float64))
    n = x.size
    F = np.clip(cdf(x), 1e-300, 1 - 1e-16)
    i = np.arange(1, n + 1)
    return float(-n - np.sum((2 * i - 1) / n * (np.log(F) + np.log1p(-F[::-1]))))


def ad_limit_cdf(z, terms=12):
    """Limiting P(A^2 <= z) of the fully specified case."""
    if z <= 0.0:
        return 0.0
    total, c = 0.0, 1.0
    for j in range(terms):
        if j > 0:
            c *= -(j - 0.5) / j                     # binom(-1/2, j)
        k = 4 * j + 1
        b = k * k * math.pi ** 2 / (8.0 * z)
        integral, _ = integrate.quad(lambda w: math.exp(z / (8.0 * (w * w + 1.0)) - b * w * w),
                                     0.0, np.inf, limit=200)
        total += c * k * math.exp(-b) * integral
    return min(1.0, max(0.0, math.sqrt(2.0 * math.pi) / z * total))


def ad_pvalue(a2):
    """p-value of A^2 = a2 (probability of a value at least as large)."""
    return 1.0 - ad_limit_cdf(a2)
