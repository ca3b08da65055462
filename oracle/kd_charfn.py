"""Exact characteristic function of the KD scheme's displacement -- TEST
INFRASTRUCTURE ONLY (part of the oracle: only tests/, the smoke check and the
CPU-baseline leg of the benchmark use it).

For the homogeneous background with mu = 0, a path of Alg. 1 on the grid
dt_l = T/n is a sequence of KD events.  From a grid point (or t = 0) a flight
of length tau = E/R starts (E ~ Exp(1)).  If it ends before T, the particle
moves ballistically for tau and then diffusively until the next grid point,
a time theta.  The diffusive move is a + d chi with a fresh velocity v' and
chi ~ N(0,1):

    a = v' (1 - e^{-s}) / R,
    d^2 = 2 sigma^2/R^2 f(s) + v'^2/R^2 g(s),   s = R theta,

(eqs. advection and diffusion, Sec. 2).  If the flight reaches T, the
particle drifts to T.  The displacement D = x(T) - x(0) is linear in every
velocity and every chi, so phi(k) = E[exp(i k D)] reduces in closed form over
them:

* chi_j gives exp(-k^2 d_j^2 / 2);
* the velocity v = sigma nu drawn at an event with diffusive time theta
  enters D as v c, with c = (1 - e^{-R theta})/R plus the following kinetic
  time (or the drift to T), and enters d^2 as v^2 g(R theta)/R^2.  For
  nu ~ N(0,1),
      E[exp(i k sigma c nu - k^2 sigma^2 g nu^2 / (2 R^2))]
          = (1 + b)^{-1/2} exp(-k^2 sigma^2 c^2 / (2 (1 + b))),
  with b = k^2 sigma^2 g / R^2.  The initial velocity has theta = 0.

What is left is an expectation over the flights.  In step units a flight is
q = E/(R dt) ~ Exp(R dt).  Its integer part sets how many grid points the
particle passes before the collision; its fractional part u sets the next
diffusive time theta' = dt (1 - u).  With r grid steps left, the remaining
factor G(r, theta) obeys

    G(r, theta) = e^{-R dt r} V(theta, w(theta) + r dt)
                + sum_{s<r} int_0^1 R dt e^{-R dt (s+u)} V(theta, w(theta) + (s+u) dt)
                               F(dt (1-u)) G(r-s-1, dt (1-u)) du,

where V is the velocity factor above, w(theta) = (1 - e^{-R theta})/R and
F(theta') = exp(-k^2 sigma^2 f(R theta')/R^2).  Then phi(k) = G(n, 0).  The
integral over u is a Gauss-Legendre rule in the variable
(1 - e^{-R dt u})/(1 - e^{-R dt}), which takes the exponential weight
exactly.  The rule is accurate while R dt stays moderate (R dt <= 5 here).

This computation shares nothing with the oracle's path simulation.  It is
checked by itself against the closed-form second moment and the ballistic
and Brownian limits.
"""
import math

import numpy as np


def _f(s):
    """f(s) = 2(e^{-s} - 1) + s(e^{-s} + 1) (eq. diffusion); Taylor series
    sum_{n>=3} (-1)^n (2 - n) s^n / n! below s = 1/2."""
    s = np.asarray(s, np.float64)
    big = s >= 0.5
    e = np.exp(-np.where(big, s, 0.0))
    closed = 2.0 * (e - 1.0) + s * (e + 1.0)
    ser = np.zeros_like(s)
    for n in range(3, 30):
        ser += (-1) ** n * (2 - n) * s ** n / math.factorial(n)
    return np.where(big, closed, ser)


def _g(s):
    """g(s) = 1 - 2 s e^{-s} - e^{-2s} (eq. diffusion); Taylor series
    sum_{n>=3} (-1)^n (2n - 2^n) s^n / n! below s = 1/2."""
    s = np.asarray(s, np.float64)
    big = s >= 0.5
    e = np.exp(-np.where(big, s, 0.0))
    closed = 1.0 - 2.0 * s * e - e * e
    ser = np.zeros_like(s)
    for n in range(3, 30):
        ser += (-1) ** n * (2 * n - 2 ** n) * s ** n / math.factorial(n)
    return np.where(big, closed, ser)


def kd_charfn(k, eps, dt, n, nodes=64):
    """E[cos(k D)] for D = x(T) - x(0) of Alg. 1 with R = 1/eps^2,
    sigma = 1/eps, mu = 0, n steps of length dt (T = n dt)."""
    R = 1.0 / (eps * eps)
    sig2 = 1.0 / (eps * eps)
    kk = k * k * sig2
    a = R * dt
    z, wz = np.polynomial.legendre.leggauss(nodes)
    w01 = 0.5 * (z + 1.0)
    mass = -math.expm1(-a)
    u = -np.log1p(-w01 * mass) / a        # fractional parts of the flight
    wu = 0.5 * wz * mass                  # weights of R dt e^{-R dt u} du
    theta_next = dt * (1.0 - u)
    F = np.exp(-kk * _f(R * theta_next) / (R * R))

    def vel(theta, c):
        b = kk * _g(R * theta) / (R * R)
        return np.exp(-kk * c * c / (2.0 * (1.0 + b))) / np.sqrt(1.0 + b)

    def G(r, theta, table):
        w = -np.expm1(-R * theta) / R
        out = math.exp(-a * r) * vel(theta, w + r * dt)
        for s in range(r):
            c = w[:, None] + (s + u[None, :]) * dt
            out = out + math.exp(-a * s) * (vel(theta[:, None], c)
                                             * (wu * F * table[r - s - 1])[None, :]).sum(axis=1)
        return out

    table = []
    for r in range(n):
        table.append(G(r, theta_next, table))
    return float(G(n, np.zeros(1), table)[0])
