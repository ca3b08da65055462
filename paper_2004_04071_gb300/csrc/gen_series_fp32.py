"""Writes the FP32 polynomial coefficients of the KD coefficient series.

For 0 <= s <= 1 the FP32 pair kernels evaluate (Sec. 2, eqs. advection and
diffusion, with e = exp(-s))
    F(s) = f(s)/s^3,  f(s) = 2(e - 1) + s(e + 1) = sum_{n>=3} (-1)^n (2 - n) s^n / n!
    G(s) = g(s)/s^3,  g(s) = 1 - 2 s e - e^2    = sum_{n>=3} (-1)^n (2n - 2^n) s^n / n!
    H(s) = h(s)/s^2,  h(s) = e + s - 1          = sum_{n>=2} (-1)^n s^n / n!
as polynomials in s.  Each polynomial interpolates its function at the
Chebyshev nodes of [0, 1] (Chebyshev economisation: near-minimax, far fewer
terms than the truncated Taylor series for the same error at s = 1).  The
function values come from the Taylor series summed to 60 terms in 40-digit
arithmetic.  The script prints the coefficients, highest degree first, and
the largest relative error of FP32 Horner evaluation with fused multiply-adds
over 4001 points of [0, 1].

    python paper_2004_04071_gb300/csrc/gen_series_fp32.py
"""
import mpmath as mp
import numpy as np

mp.mp.dps = 40

SERIES = {
    # name: (coefficient of s^n, first n, degree)
    "F": (lambda n: mp.mpf((-1) ** n * (2 - n)) / mp.factorial(n), 3, 6),
    "G": (lambda n: mp.mpf((-1) ** n * (2 * n - 2 ** n)) / mp.factorial(n), 3, 9),
    "H": (lambda n: mp.mpf((-1) ** n) / mp.factorial(n), 2, 6),
}


def value(coef, n0, s, terms=60):
    return mp.fsum(coef(n) * s ** (n - n0) for n in range(n0, n0 + terms))


def chebyshev_interpolant(f, deg):
    """Monomial coefficients (lowest first) of the degree-deg polynomial that
    interpolates f at the Chebyshev nodes of [0, 1]."""
    nodes = [mp.mpf(1) / 2 + mp.cos(mp.pi * (k + mp.mpf(1) / 2) / (deg + 1)) / 2 for k in range(deg + 1)]
    V = mp.matrix([[x ** j for j in range(deg + 1)] for x in nodes])
    c = mp.lu_solve(V, mp.matrix([f(x) for x in nodes]))
    return [c[j] for j in range(deg + 1)]


def horner_fp32(c32, x):
    p = c32[-1]
    for c in reversed(c32[:-1]):
        p = np.float32(float(p) * float(x) + float(c))   # one rounding, as an FMA
    return p


def main():
    grid = [mp.mpf(i) / 4000 for i in range(4001)]
    for name, (coef, n0, deg) in SERIES.items():
        f = lambda s: value(coef, n0, s)
        c32 = [np.float32(float(c)) for c in chebyshev_interpolant(f, deg)]
        err = max(abs(float(horner_fp32(c32, np.float32(float(x)))) - float(f(x))) / abs(float(f(x)))
                  for x in grid)
        print("%s: degree %d, max relative error %.2e (%.2f x 2^-24)" % (name, deg, err, err / 2.0 ** -24))
        print("    " + ", ".join("%.9ef" % c for c in reversed(c32)))


if __name__ == "__main__":
    main()
