"""Scalar monitors of a nodal field (no counterpart in the paper's equations except as noted).

* mass   = 1^T M U with M the assembled Q1 mass matrix (applied through its 1D factors A_a, the
           Kronecker structure of eq. (4.1), which the tests pin against global assembly).
* energy = 1/2 U^T K U + sum over interior nodes of prod_a h_a * (u^2 - 1)^2 / 4; the paper states an
           energy only for the Flory-Huggins case (Section 5.2), so this lumped double-well form is
           a reading for f = u - u^3 and is used as a monitor only (the quadratic term is pinned
           through K, the potential through its reaction: dE/du = -f on constant periodic fields,
           zero in the wells).
* maxabs = max |u|, the quantity of the maximum bound principle discussed in Sections 1 and 5.2.

With ``flory_huggins=(theta, theta_c)`` the potential term is that of the energy functional stated
for Example 5.3 (Section 5.2), (theta/2)((1+u) ln(1+u) + (1-u) ln(1-u)) - (theta_c/2) u^2, taken by
the same nodal (lumped) quadrature (a reading: the paper does not say how it evaluates the
integral), and the gradient term 1/2 U^T K U with K = eps^2 (...) is exact for the finite element
function (D = eps^2). Periodic fields (``bc='periodic'``) use the periodic assembly.
``fh_max_bound`` is the maximum bound gamma of Example 5.3: the positive root of f, found by
bisection.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

from .etd import mode_product
from .fem import assemble_1d


def fh_max_bound(theta: float, theta_c: float) -> float:
    """Positive root of (theta/2) ln((1-u)/(1+u)) + theta_c u on (0, 1) (theta < theta_c)."""
    f = lambda u: 0.5 * theta * np.log((1.0 - u) / (1.0 + u)) + theta_c * u
    lo, hi = 1e-6, 1.0 - 1e-15          # f(lo) > 0 > f(hi) when theta < theta_c
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def monitors(U: np.ndarray, N: Sequence[int], h: Sequence[float], D: float, bc: str = "dirichlet",
             flory_huggins: tuple | None = None) -> dict:
    d = len(N)
    AB = [assemble_1d(int(n), float(hh), bc) for n, hh in zip(N, h)]
    MU = U
    for a in range(d):
        MU = mode_product(AB[a][0], MU, a)
    KU = np.zeros_like(U)
    for a in range(d):
        T = U
        for b in range(d):
            T = mode_product(AB[b][1] if b == a else AB[b][0], T, b)
        KU = KU + D * T
    cell = float(np.prod(h))
    if flory_huggins is None:
        pot = 0.25 * np.sum((U * U - 1.0) ** 2)
    else:
        theta, theta_c = flory_huggins
        pot = np.sum(0.5 * theta * ((1.0 + U) * np.log(1.0 + U) + (1.0 - U) * np.log(1.0 - U))
                     - 0.5 * theta_c * U * U)
    return {
        "mass": float(MU.sum()),
        "energy": float(0.5 * np.sum(U * KU) + cell * pot),
        "maxabs": float(np.max(np.abs(U))) if U.size else 0.0,
        "nonfinite": int(np.count_nonzero(~np.isfinite(U))),
    }
