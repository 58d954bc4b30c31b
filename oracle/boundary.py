"""Nonhomogeneous Dirichlet data (Section 4: the given boundary values of the solution enter the
scheme as part of f; Example 5.2 of Section 5 is of this form).

Reading: the interior rows of the Galerkin system on all nodes, with the boundary nodal values g(t)
prescribed and the reaction taken on nodal values of every node (the group finite element reading
F = M f(u) of the homogeneous case):
    M_II U' + K_II U = M_II f(U) + b(t),   b(t) = M_IB (f(g) - g'(t)) - K_IB g(t),
so the EIFE schemes of Section 2 run unchanged on U with the time-dependent reaction
    f~(t, U) = f(t, U) + M_II^{-1} b(t).
M and K come from the 1D matrices on all nodes (Kronecker structure of eq. (4.1)); M_II^{-1} is
applied by dense solves with the interior 1D mass matrix along each axis.
Parity: pinned (a discrete harmonic state stays; a constant root of f stays; convergence at orders
1 and 2 to a library ODE solve of the globally assembled system; the printed temporal L2 errors of
Table 4 (Example 5.2) approached on refined meshes).
"""
from __future__ import annotations

from typing import Callable, Sequence

import numpy as np

from .etd import mode_product
from .fem import assemble_1d_all_nodes

# g(t) -> (values, time derivatives) on the full node grid, shape (N_z+1, N_y+1, N_x+1) or
# (N_y+1, N_x+1); only the boundary entries are read.
BoundaryData = Callable[[float], tuple]


def boundary_mask(N: Sequence[int]) -> np.ndarray:
    """True on boundary nodes of the full node grid (storage order z, y, x)."""
    shape = tuple(int(n) + 1 for n in reversed(N))
    m = np.ones(shape, dtype=bool)
    m[tuple(slice(1, -1) for _ in shape)] = False
    return m


def boundary_source(N: Sequence[int], h: Sequence[float], D: float, f: Callable, data: BoundaryData):
    """t -> M_II^{-1} b(t) on the interior nodes (storage order z, y, x)."""
    d = len(N)
    AB = [assemble_1d_all_nodes(int(n), float(hh)) for n, hh in zip(N, h)]
    Ainv = [np.linalg.inv(A[1:-1, 1:-1]) for A, _ in AB]
    mask = boundary_mask(N)
    inner = tuple(slice(1, -1) for _ in range(d))

    def src(t: float) -> np.ndarray:
        g, gdot = data(t)
        g = np.where(mask, np.asarray(g, dtype=np.float64), 0.0)
        gdot = np.where(mask, np.asarray(gdot, dtype=np.float64), 0.0)
        r = np.where(mask, f(t, g), 0.0) - gdot
        Mr = r
        for a in range(d):
            Mr = mode_product(AB[a][0], Mr, a)
        Kg = np.zeros_like(g)
        for a in range(d):
            T = g
            for b in range(d):
                T = mode_product(AB[b][1] if b == a else AB[b][0], T, b)
            Kg = Kg + D * T
        b_int = (Mr - Kg)[inner]
        for a in range(d):
            b_int = mode_product(Ainv[a], b_int, a)
        return b_int

    return src


def with_boundary(f: Callable, src: Callable) -> Callable:
    """f~(t, U) = f(t, U) + M_II^{-1} b(t)."""
    def ft(t, U):
        return f(t, U) + src(t)
    return ft
