"""Pins for the oracle's phi-functions (Section 2.2) against 50-digit values."""
import math

import mpmath
import numpy as np
import pytest

from oracle.phi import phi

mpmath.mp.dps = 50


def _phi_mp(k, z):
    """phi_k from its Taylor series sum_m z^m / (m + k)! at 50 digits (no cancellation)."""
    z = mpmath.mpf(z)
    s, term, m = mpmath.mpf(0), mpmath.mpf(1) / mpmath.factorial(k), 0
    while True:
        s += term
        m += 1
        term = term * z / (m + k)
        if abs(term) < mpmath.mpf(10) ** -45 * max(abs(s), mpmath.mpf(1)) and m > abs(z) + 5:
            break
    return s


ZS = [0.0, 1e-14, -1e-12, 1e-8, -1e-5, 3e-4, -0.01, 0.3, -0.5, -0.999, 1.0, -1.0, -1.001, 1.5,
      -2.0, -7.3, -23.6, -60.0, 4.0]


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_phi_against_50_digit_series(k):
    got = phi(k, np.array(ZS))
    for z, g in zip(ZS, got):
        ref = float(_phi_mp(k, z))
        # the recurrence for |z| just above 1 loses a few bits for k = 3
        assert g == pytest.approx(ref, rel=3e-14 if k < 3 else 1e-12), (k, z)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_phi_at_zero_is_inverse_factorial(k):
    assert float(phi(k, 0.0)) == pytest.approx(1.0 / math.factorial(k), rel=1e-15)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_phi_recurrence_relation(k):
    """phi_{k+1}(z) = (phi_k(z) - phi_k(0)) / z away from z = 0."""
    z = np.array([-3.0, -1.5, -0.7, 0.4, 2.0])
    lhs = phi(k + 1, z)
    rhs = (phi(k, z) - float(phi(k, 0.0))) / z
    np.testing.assert_allclose(lhs, rhs, rtol=1e-13)


def test_phi_continuous_across_method_switch():
    eps = 1e-9
    for k in (1, 2):
        for s in (-1.0, 1.0):
            a, b = phi(k, np.array([s * (1 - eps), s * (1 + eps)]))
            assert abs(a - b) < 1e-8
