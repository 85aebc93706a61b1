"""Fit of the scaled complementary error function used by the mixed-form
real-space Ewald sum (csrc/common.cuh, erfc_scaled_fit):

    erfc(x) = exp(-x^2) t P(t),   t = 1 / (1 + x / 2),   0 <= x <= 4.1,

P of degree 8, a Chebyshev least-squares fit (relative weighting) of
erfc(x) exp(x^2) / t on 40001 points, converted to monomials in t.  4.1 covers
kappa r up to the FP32-level cutoff (kappa = 5 / L, r <= 0.8 L gives 4).

`python -m paper_1605_08423_gb300.fit_erfc` prints the coefficients (lowest
order first) and the relative error of their FP32 Horner evaluation.
"""
from __future__ import annotations

import numpy as np

X_MAX = 4.1
DEGREE = 8


def _target(x):
    from scipy.special import erfc
    return erfc(x) * np.exp(x * x)


def fit(degree: int = DEGREE, n: int = 40001) -> np.ndarray:
    xs = np.linspace(0.0, X_MAX, n)
    t = 1.0 / (1.0 + 0.5 * xs)
    tmin = t.min()
    u = (2.0 * t - (1.0 + tmin)) / (1.0 - tmin)
    g = _target(xs)
    c = np.polynomial.chebyshev.chebfit(u, g / t, degree, w=t / g)
    p_u = np.polynomial.Polynomial(np.polynomial.chebyshev.cheb2poly(c))
    a, b = 2.0 / (1.0 - tmin), -(1.0 + tmin) / (1.0 - tmin)
    return p_u(np.polynomial.Polynomial([b, a])).coef


def fp32_max_rel_error(coef, n: int = 40001) -> float:
    """Largest relative error of e t P(t) evaluated as the kernel does (FP32
    Horner, FP32 t), against erfc(x) exp(x^2) in FP64."""
    xs = np.linspace(0.0, X_MAX, n)
    x32 = xs.astype(np.float32)
    t32 = (np.float32(1.0) / (np.float32(1.0) + np.float32(0.5) * x32)).astype(np.float32)
    c32 = [np.float32(v) for v in coef]
    acc = c32[-1]
    for cc in c32[-2::-1]:
        acc = (acc * t32 + cc).astype(np.float32)
    approx = (acc * t32).astype(np.float64)
    g = _target(xs)
    return float(np.max(np.abs(approx - g) / g))


if __name__ == "__main__":
    cf = fit()
    print([f"{float(np.float32(v)):.9e}" for v in cf])
    print("max relative error (FP32 evaluation):", fp32_max_rel_error(cf))
