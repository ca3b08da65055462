"""Write periodic_benchmark_exact.json: the exact int x^2 f that the periodic
benchmark problem's estimate targets, for eps in {1, 0.1, 1e-3}.

The MLMC estimate targets E[F(x_L)] at the finest level L.  With
x_0 ~ 1 + cos 2 pi x and F(x) = (x mod 1)^2 that is
1/3 + phi_L(2 pi)/(2 pi^2), phi_L from the exact characteristic function of
the KD scheme (kd_charfn).  At eps = 1e-3 the finest level has 8192 steps with
R dt = 122, beyond the dynamic program's quadrature.  There the scheme's
displacement has variance 2(T - eps^2(1 - e^{-T/eps^2})) ~ 2 and is a sum of
thousands of nearly Gaussian increments, so phi(2 pi) ~ e^{-4 pi^2} < 1e-12,
and the value is taken as 1/3.

Run from the repository root: python tests/golden/make_periodic_exact.py
"""
import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle.kd_charfn import kd_charfn  # noqa: E402


def main():
    out = {"qoi": "int x^2 f at T = 1, finest level of the periodic benchmark problem",
           "values": []}
    for eps in W.PERIODIC_EPS:
        d = W.periodic_problem(eps)
        L = d["L"]
        dt = d["dt0"] / d["M"] ** L
        n = int(round(d["T"] / dt))
        if eps >= 0.1:
            phi = kd_charfn(2 * math.pi, eps, dt, n)
            how = "kd_charfn, %d steps" % n
        else:
            phi = 0.0
            how = "Brownian limit, |phi(2 pi)| < 1e-12"
        out["values"].append({"eps": eps, "L": L, "phi_2pi": phi,
                              "exact": 1.0 / 3.0 + phi / (2 * math.pi ** 2), "how": how})
    with open(os.path.join(HERE, "periodic_benchmark_exact.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
