"""The orthonormal DST-I along one axis, written from its definition (Section 4), and the
orthonormal discrete Hartley transform used for periodic axes.

S_ij = sqrt(2/N) sin(i j pi / N), i, j = 1..N-1 (the sine matrix P of Section 4 scaled to be
orthonormal: Section 4 calls P orthogonal, but P P^T = (N/2) I); S is symmetric and S S = I, so it is both the forward
transform U~ = S^T (x)_a U and its inverse. Applied as a dense product along the axis.
Parity: pinned (equals, up to sign, the numerically computed eigenvectors of A and B; S S = I).

Periodic axes: H_jk = N^{-1/2} cas(2 pi j k / N), cas t = cos t + sin t, j, k = 0..N-1; H is
symmetric, H H = I, and diagonalises the circulant A and B of the periodic case (whose eigenvalues
depend on cos(2 pi k / N) only), so it serves as the real form of the DFT of Section 4's remarks on
periodic boundaries. Parity: pinned (H = Re F - Im F for the library FFT F; H H = I; H A H
diagonal with the closed-form eigenvalues).
"""
from __future__ import annotations

import numpy as np

from .etd import mode_product


def sine_matrix(N: int) -> np.ndarray:
    """sqrt(2/N) sin(pi i j / N); i j is reduced modulo 2N first (exact integer arithmetic, the
    sine has period 2N in i j), so the angle stays below 2 pi and carries no large rounding error."""
    i = np.arange(1, N)
    ij = np.outer(i, i) % (2 * N)
    return np.sqrt(2.0 / N) * np.sin(ij * np.pi / N)


def dst_axis(U: np.ndarray, axis: int) -> np.ndarray:
    """S (x)_axis U for paper axis ``axis`` (0 = x, the last array axis)."""
    U = np.asarray(U, dtype=np.float64)
    N = U.shape[U.ndim - 1 - axis] + 1
    return mode_product(sine_matrix(N), U, axis)


def hartley_matrix(N: int) -> np.ndarray:
    """N^{-1/2} (cos + sin)(2 pi j k / N), j k reduced modulo N first (exact integer arithmetic)."""
    j = np.arange(N)
    t = 2.0 * np.pi * (np.outer(j, j) % N) / N
    return (np.cos(t) + np.sin(t)) / np.sqrt(N)


def dht_axis(U: np.ndarray, axis: int) -> np.ndarray:
    """H (x)_axis U for paper axis ``axis`` (0 = x, the last array axis) of a periodic field."""
    U = np.asarray(U, dtype=np.float64)
    return mode_product(hartley_matrix(U.shape[U.ndim - 1 - axis]), U, axis)
