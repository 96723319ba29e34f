"""Partial-fraction coefficients of rational approximations, inputs to the rational-function
application r(A) b = alpha0 b + sum_s alpha_s (A + sigma_s)^-1 b.

The paper uses such approximations in RHMC but prints no coefficients; these are generated here
for the tests and benchmarks and handed to both the GPU library and the oracle as inputs.

inv_sqrt(n, lo, hi): r(lambda) ~ lambda^(-1/2) on [lo, hi] from the integral representation
  lambda^(-1/2) = (2/pi) int_0^inf dt / (lambda + t^2),
substituted t = exp(u) and discretised by the trapezoidal (sinc) rule, which converges
exponentially for such analytic integrands (Hale, Higham and Trefethen, "Computing A^alpha,
log(A), and related matrix functions by contour integrals", SIAM J. Numer. Anal. 46 (2008)):
  sigma_k = exp(2 u_k),  alpha_k = (2/pi) h exp(u_k),  u_k = u_min + k h,  k = 0 .. n-1.
The window [u_min, u_max] and the step h follow from the spectrum bounds; alpha0 = 0.
"""
from __future__ import annotations

import math


def inv_sqrt(n: int, lo: float, hi: float):
    """(alpha0, alpha[n], sigma[n]) with sum_k alpha_k / (lambda + sigma_k) ~ lambda^(-1/2)."""
    if n < 2 or not (0.0 < lo < hi):
        raise ValueError("need n >= 2 and 0 < lo < hi")
    # the integrand e^u / (lambda + e^(2u)) decays as e^u below u = log(sqrt(lambda)) and as
    # lambda e^(-u) above: cover [log sqrt(lo) - L, log sqrt(hi) + L] with tails below ~e^-L
    u_lo = 0.5 * math.log(lo)
    u_hi = 0.5 * math.log(hi)
    # errors relative to lambda^(-1/2): truncating L beyond the window costs about e^-L; the
    # trapezoidal rule with step h costs about e^(-pi^2 / (2 h)) (the integrand's poles lie at
    # imaginary part pi/2).  L = pi^2 / (2 h) and W + 2 L = (n - 1) h, with W = u_hi - u_lo.
    w = u_hi - u_lo
    h = (w + math.sqrt(w * w + 4.0 * math.pi ** 2 * (n - 1))) / (2.0 * (n - 1))
    tail = math.pi ** 2 / (2.0 * h)
    u0 = u_lo - tail
    alpha, sigma = [], []
    for k in range(n):
        u = u0 + k * h
        sigma.append(math.exp(2.0 * u))
        alpha.append(2.0 / math.pi * h * math.exp(u))
    return 0.0, alpha, sigma


def evaluate(alpha0: float, alpha, sigma, lam: float) -> float:
    """r(lambda) = alpha0 + sum_k alpha_k / (lambda + sigma_k)."""
    return alpha0 + sum(a / (lam + s) for a, s in zip(alpha, sigma))
