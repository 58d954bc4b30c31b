"""Simultaneous diagonalisation of the 1D mass and stiffness matrices (Section 4).

A and B share an orthogonal eigenvector matrix P: A = P Lambda_A P^T, B = P Lambda_B P^T.
The oracle finds P numerically (library symmetric eigensolver applied to A) and reads
Lambda_B = P^T B P off the diagonal; it does not use the closed-form sines or eigenvalues, which
are pins in the tests. The per-mode rate of one axis is mu_i = Lambda_B,ii / Lambda_A,ii, and the
multi-axis rate of eq. (4.3) is h_ijk = D (mu_x,i + mu_y,j + mu_z,k) (the tensor H of Section 4).
Periodic case (Section 4, closing remarks): A and B are circulant; the same numerical route applies
(eigenvalues come in pairs, and within each two-dimensional eigenspace of A the matrix B is a
multiple of the identity, so any orthonormal basis of it that eigh returns also diagonalises B).
Parity: pinned (closed forms of the corrected eigenvalues, both cases; P^T B P diagonal; S^2 = I
for the sine matrix; the periodic step against one computed with the library FFT).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .fem import assemble_1d


@dataclass
class AxisEigen:
    P: np.ndarray        # (n, n) orthonormal (n = N-1 Dirichlet, N periodic); column i is an eigenvector
    lamA: np.ndarray     # eigenvalues of A
    lamB: np.ndarray     # diagonal of P^T B P
    mu: np.ndarray       # lamB / lamA
    offdiag: float       # max |off-diagonal| of P^T B P (simultaneous diagonalisation check)


def axis_eigen(N: int, h: float, bc: str = "dirichlet") -> AxisEigen:
    A, B = assemble_1d(N, h, bc)
    lamA, P = np.linalg.eigh(A)
    PBP = P.T @ B @ P
    lamB = np.diag(PBP).copy()
    off = float(np.max(np.abs(PBP - np.diag(lamB)))) if PBP.size > 1 else 0.0
    return AxisEigen(P=P, lamA=lamA, lamB=lamB, mu=lamB / lamA, offdiag=off)


def mode_rates(mus: list, D: float) -> np.ndarray:
    """h_{ijk} = D * sum_a mu_a over all modes; array axes in storage order (z, y, x).

    ``mus`` is per axis, x first.
    """
    d = len(mus)
    lam = np.zeros(tuple(len(m) for m in reversed(mus)))
    for a, m in enumerate(mus):
        shape = [1] * d
        shape[d - 1 - a] = len(m)
        lam = lam + np.asarray(m).reshape(shape)
    return D * lam
