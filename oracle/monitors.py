"""Scalar monitors of a nodal field (no counterpart in the paper's equations except as noted).

* mass   = 1^T M U with M the assembled Q1 mass matrix (applied through its 1D factors A_a, the
           Kronecker structure of eq. (4.1), which the tests pin against global assembly).
* energy = 1/2 U^T K U + sum over interior nodes of prod_a h_a * (u^2 - 1)^2 / 4; the paper states an
           energy only for the Flory-Huggins case (Section 5.2), so this lumped double-well form is
           a reading for f = u - u^3 and is used as a monitor only (parity unpinned for its
           potential term; the quadratic term is pinned through K).
* maxabs = max |u|, the quantity of the maximum bound principle discussed in Sections 1 and 5.2.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

from .etd import mode_product
from .fem import assemble_1d


def monitors(U: np.ndarray, N: Sequence[int], h: Sequence[float], D: float) -> dict:
    d = len(N)
    AB = [assemble_1d(int(n), float(hh)) for n, hh in zip(N, h)]
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
    return {
        "mass": float(MU.sum()),
        "energy": float(0.5 * np.sum(U * KU) + cell * 0.25 * np.sum((U * U - 1.0) ** 2)),
        "maxabs": float(np.max(np.abs(U))) if U.size else 0.0,
        "nonfinite": int(np.count_nonzero(~np.isfinite(U))),
    }
