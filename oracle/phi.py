"""phi-functions of the exponential Runge-Kutta weights (Section 2.2).

phi_k(z) = int_0^1 exp((1 - theta) z) theta^(k-1) / (k-1)! dtheta for k >= 1, phi_0(z) = exp(z).

* |z| <= 1: Gauss-Legendre quadrature of the defining integral with 24 nodes on [0, 1]; the
  integrand is entire, so the rule is exact to rounding for these z.
* |z| > 1: the recurrence phi_{k+1}(z) = (phi_k(z) - phi_k(0)) / z with phi_k(0) = 1/k!, started
  from phi_0 = exp(z); no cancellation worth the name happens for |z| > 1 and k <= 3.
Parity: pinned (50-digit values of the closed form, phi_k(0) = 1/k!, the recurrence).
"""
from __future__ import annotations

import math

import numpy as np

_GL_X, _GL_W = np.polynomial.legendre.leggauss(24)
_THETA = 0.5 * (_GL_X + 1.0)
_WEIGHT = 0.5 * _GL_W


def _phi_quadrature(k: int, z: np.ndarray) -> np.ndarray:
    kern = _THETA ** (k - 1) / math.factorial(k - 1)
    return np.exp(np.multiply.outer(z, 1.0 - _THETA)) @ (_WEIGHT * kern)


def _phi_recurrence(k: int, z: np.ndarray) -> np.ndarray:
    p = np.exp(z)
    for j in range(k):
        p = (p - 1.0 / math.factorial(j)) / z
    return p


def phi(k: int, z) -> np.ndarray:
    """phi_k(z) for real z (scalar or array), FP64."""
    z = np.asarray(z, dtype=np.float64)
    if k == 0:
        return np.exp(z)
    out = np.empty_like(z)
    small = np.abs(z) <= 1.0
    if np.any(small):
        out[small] = _phi_quadrature(k, z[small])
    if np.any(~small):
        out[~small] = _phi_recurrence(k, z[~small])
    return out
