"""Q1 (multilinear) finite elements on a uniform rectangular mesh, homogeneous Dirichlet or periodic.

Section 2.1: V_h is the tensor product of 1D continuous piecewise-linear spaces with nodes
x^j = a + j h, j = 0..N, and only the N-1 interior hat functions kept (eq. (2.4)).
Periodic case (Section 4, closing remarks): node N is node 0, so the N hat functions
j = 0..N-1 are kept and element N-1 joins node N-1 to node 0.
Section 4, eq. (4.1): the semi-discrete system is M dU/dt + K U = F with
M = A_x (x) A_y (x) A_z, K = D (B_x (x) A_y (x) A_z + ...), A = (h/6) R, B = (1/h) G^D.

Here A, B, M and K are assembled from element integrals (eq. (2.5) tested with every basis
function), never from the Kronecker form; the Kronecker form is a pin in the tests.
Parity: pinned (element integrals against Gauss quadrature of the hat functions; assembled
matrices against eq. (4.1)).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp


def element_mass_1d(h: float) -> np.ndarray:
    """Integrals of products of the two linear shape functions on an element of length h.

    int_0^h (1 - s/h)^2 ds = h/3 and int_0^h (1 - s/h)(s/h) ds = h/6.
    """
    return np.array([[h / 3.0, h / 6.0], [h / 6.0, h / 3.0]])


def element_stiffness_1d(h: float) -> np.ndarray:
    """Integrals of products of the derivatives (-1/h and +1/h) of the two shape functions."""
    return np.array([[1.0 / h, -1.0 / h], [-1.0 / h, 1.0 / h]])


def _check_bc(bc: str) -> None:
    if bc not in ("dirichlet", "periodic"):
        raise ValueError("bc must be 'dirichlet' or 'periodic'")


def assemble_1d(N: int, h: float, bc: str = "dirichlet") -> tuple[np.ndarray, np.ndarray]:
    """Assemble the 1D mass A and stiffness B over N elements.

    Dirichlet: keep the N-1 interior nodes, dense (N-1) x (N-1). Node j of element e is e + j.
    Periodic: node j of element e is (e + j) mod N, dense N x N (N >= 3, so that the two nodes of
    an element are distinct and no element meets itself).
    """
    _check_bc(bc)
    if N < 2 or (bc == "periodic" and N < 3):
        raise ValueError("too few intervals")
    me, ke = element_mass_1d(h), element_stiffness_1d(h)
    if bc == "periodic":
        A = np.zeros((N, N))
        B = np.zeros((N, N))
        for e in range(N):
            nodes = (e, (e + 1) % N)
            for a in range(2):
                for b in range(2):
                    A[nodes[a], nodes[b]] += me[a, b]
                    B[nodes[a], nodes[b]] += ke[a, b]
        return A, B
    Af = np.zeros((N + 1, N + 1))
    Bf = np.zeros((N + 1, N + 1))
    for e in range(N):
        for a in range(2):
            for b in range(2):
                Af[e + a, e + b] += me[a, b]
                Bf[e + a, e + b] += ke[a, b]
    return Af[1:N, 1:N].copy(), Bf[1:N, 1:N].copy()


def assemble_1d_all_nodes(N: int, h: float) -> tuple[np.ndarray, np.ndarray]:
    """The 1D mass and stiffness over N elements on all N+1 nodes (boundary rows included), as
    needed for nonhomogeneous Dirichlet data: the interior rows couple the interior unknowns to the
    prescribed boundary values through the columns of nodes 0 and N."""
    if N < 2:
        raise ValueError("need at least two intervals")
    A = np.zeros((N + 1, N + 1))
    B = np.zeros((N + 1, N + 1))
    me, ke = element_mass_1d(h), element_stiffness_1d(h)
    for e in range(N):
        for a in range(2):
            for b in range(2):
                A[e + a, e + b] += me[a, b]
                B[e + a, e + b] += ke[a, b]
    return A, B


def element_matrices_nd(h: tuple, D: float) -> tuple[np.ndarray, np.ndarray]:
    """Q1 element mass and stiffness in d dimensions (local nodes ordered x fastest).

    The basis functions on an element are products of 1D shape functions, so each integral over
    the element factorises into 1D integrals:
      mass:      prod_a m_a[i_a, j_a]
      stiffness: D * sum_a k_a[i_a, j_a] * prod_{b != a} m_b[i_b, j_b]   (bilinear form (2.3))
    """
    d = len(h)
    m1 = [element_mass_1d(ha) for ha in h]
    k1 = [element_stiffness_1d(ha) for ha in h]
    nloc = 2 ** d
    locs = [tuple((n >> a) & 1 for a in range(d)) for n in range(nloc)]  # a = 0 is x (fastest)
    Me = np.zeros((nloc, nloc))
    Ke = np.zeros((nloc, nloc))
    for p, ip in enumerate(locs):
        for q, iq in enumerate(locs):
            Me[p, q] = np.prod([m1[a][ip[a], iq[a]] for a in range(d)])
            Ke[p, q] = D * sum(
                k1[a][ip[a], iq[a]] * np.prod([m1[b][ip[b], iq[b]] for b in range(d) if b != a])
                for a in range(d))
    return Me, Ke


def assemble_global_all_nodes(N: tuple, h: tuple, D: float) -> tuple[sp.csr_matrix, sp.csr_matrix, np.ndarray]:
    """Global M and K over all (N_x+1)(N_y+1)[(N_z+1)] nodes (x fastest) and the indices of the
    interior nodes among them, from the element matrices (no Kronecker form)."""
    d = len(N)
    Me, Ke = element_matrices_nd(h, D)
    full = [n + 1 for n in N]
    strides = [int(np.prod(full[:a])) for a in range(d)]
    rows, cols, mv, kv = [], [], [], []
    locs = [tuple((n >> a) & 1 for a in range(d)) for n in range(2 ** d)]
    for e in itertools.product(*[range(n) for n in reversed(N)]):
        e = tuple(reversed(e))
        nodes = [sum((e[a] + lp[a]) * strides[a] for a in range(d)) for lp in locs]
        for p in range(len(nodes)):
            for q in range(len(nodes)):
                rows.append(nodes[p])
                cols.append(nodes[q])
                mv.append(Me[p, q])
                kv.append(Ke[p, q])
    ntot = int(np.prod(full))
    interior = []
    for idx in itertools.product(*[range(1, n) for n in reversed(N)]):
        idx = tuple(reversed(idx))
        interior.append(sum(idx[a] * strides[a] for a in range(d)))
    return (sp.coo_matrix((mv, (rows, cols)), shape=(ntot, ntot)).tocsr(),
            sp.coo_matrix((kv, (rows, cols)), shape=(ntot, ntot)).tocsr(), np.array(interior))


def assemble_global(N: tuple, h: tuple, D: float, bc: str = "dirichlet") -> tuple[sp.csr_matrix, sp.csr_matrix]:
    """Assemble the global M and K over all Q1 elements.

    N, h are per axis (x first). Dirichlet: restrict to interior nodes, numbered x fastest, matching
    the array layout (N_z-1, N_y-1, N_x-1) in C order. Periodic: node indices wrap modulo N_a, and
    the N_x N_y [N_z] unknowns match the layout (N_z, N_y, N_x).
    """
    _check_bc(bc)
    d = len(N)
    if bc == "periodic":
        if min(N) < 3:
            raise ValueError("too few intervals")
        Me, Ke = element_matrices_nd(h, D)
        strides = [int(np.prod(N[:a])) for a in range(d)]
        rows, cols, mv, kv = [], [], [], []
        locs = [tuple((n >> a) & 1 for a in range(d)) for n in range(2 ** d)]
        for e in itertools.product(*[range(n) for n in reversed(N)]):
            e = tuple(reversed(e))
            nodes = [sum(((e[a] + lp[a]) % N[a]) * strides[a] for a in range(d)) for lp in locs]
            for p in range(len(nodes)):
                for q in range(len(nodes)):
                    rows.append(nodes[p])
                    cols.append(nodes[q])
                    mv.append(Me[p, q])
                    kv.append(Ke[p, q])
        ntot = int(np.prod(N))
        return (sp.coo_matrix((mv, (rows, cols)), shape=(ntot, ntot)).tocsr(),
                sp.coo_matrix((kv, (rows, cols)), shape=(ntot, ntot)).tocsr())
    Me, Ke = element_matrices_nd(h, D)
    full = [n + 1 for n in N]
    strides = [int(np.prod(full[:a])) for a in range(d)]
    rows, cols, mv, kv = [], [], [], []
    locs = [tuple((n >> a) & 1 for a in range(d)) for n in range(2 ** d)]
    for e in itertools.product(*[range(n) for n in reversed(N)]):
        e = tuple(reversed(e))  # e[0] is the x element index
        nodes = [sum((e[a] + lp[a]) * strides[a] for a in range(d)) for lp in locs]
        for p in range(len(nodes)):
            for q in range(len(nodes)):
                rows.append(nodes[p])
                cols.append(nodes[q])
                mv.append(Me[p, q])
                kv.append(Ke[p, q])
    ntot = int(np.prod(full))
    Mf = sp.coo_matrix((mv, (rows, cols)), shape=(ntot, ntot)).tocsr()
    Kf = sp.coo_matrix((kv, (rows, cols)), shape=(ntot, ntot)).tocsr()
    interior = []
    for idx in itertools.product(*[range(1, n) for n in reversed(N)]):
        idx = tuple(reversed(idx))
        interior.append(sum(idx[a] * strides[a] for a in range(d)))
    interior = np.array(interior)
    return Mf[interior][:, interior].tocsr(), Kf[interior][:, interior].tocsr()
