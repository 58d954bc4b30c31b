"""Pins for the oracle's nonhomogeneous Dirichlet path (Section 4: boundary values of the solution
enter the scheme as part of f; Example 5.2 and Table 4 of Section 5).

The references do not go through `oracle.boundary`'s formula: discrete steady states (a linear field
is discrete-harmonic for Q1; a constant root of f), a library stiff ODE solve of the globally
assembled system with the boundary nodes prescribed (convergence orders 1 and 2 of the two
schemes), and the printed temporal L2 errors of Table 4.
"""
import math
import os

import numpy as np
import pytest
import scipy.integrate

from oracle import boundary, etd, fem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table4_example52_temporal.txt")


def _grid(N, h):
    """Full-grid node coordinates, storage order (z, y, x)."""
    axes = [np.arange(n + 1) * hh for n, hh in zip(N, h)]
    return np.meshgrid(*reversed(axes), indexing="ij")[::-1]   # X, Y[, Z]


@pytest.mark.parametrize("N,h", [((6, 5), (1 / 6, 0.2)), ((4, 5, 3), (0.25, 0.2, 1 / 3))])
@pytest.mark.parametrize("scheme", [1, 2])
def test_linear_field_is_a_discrete_steady_state(N, h, scheme):
    """f = 0 and g = a + b x + c y (+ d z): Q1 reproduces linear functions, whose interior rows of K
    vanish against the prescribed boundary, so the field stays (any tau)."""
    C = _grid(N, h)
    lin = 0.3 + 1.1 * C[0] - 0.7 * C[1] + (0.4 * C[2] if len(N) == 3 else 0.0)
    data = lambda t: (lin, np.zeros_like(lin))
    f = etd.allen_cahn(0.0, 0.0)
    src = boundary.boundary_source(N, h, 0.8, f, data)
    inner = tuple(slice(1, -1) for _ in N)
    U = etd.make_stepper(N, h, 0.8, 0.37, scheme).run(lin[inner].copy(), 4, boundary.with_boundary(f, src))
    np.testing.assert_allclose(U, lin[inner], rtol=0, atol=1e-12)


def test_constant_root_of_f_stays():
    N, h = (8, 6, 4), (1 / 8, 1 / 6, 0.25)
    one = np.ones(tuple(n + 1 for n in reversed(N)))
    f = etd.allen_cahn(1.0, -1.0)
    src = boundary.boundary_source(N, h, 1.0, f, lambda t: (one, 0 * one))
    U = etd.make_stepper(N, h, 1.0, 0.1, 2).run(np.ones((3, 5, 7)), 5, boundary.with_boundary(f, src))
    np.testing.assert_allclose(U, 1.0, rtol=0, atol=1e-13)


# ---------------------------------------------------------------- Example 5.2
EPS = 0.05
SPEED = 3 / (math.sqrt(2) * EPS)
T_END = 3 * math.sqrt(2) * EPS / 5
LEN = (math.sqrt(2), 1 / 8, 1 / 8)


def _wave(t, x):
    return 0.5 * (1 - np.tanh((x - SPEED * t) / (2 * math.sqrt(2) * EPS)))


def _wave_t(t, x):
    xi = (x - SPEED * t) / (2 * math.sqrt(2) * EPS)
    return SPEED / (4 * math.sqrt(2) * EPS) / np.cosh(xi) ** 2


def _example52(N, NT, scheme, T=T_END):
    """EIFE run of Example 5.2 on mesh N; returns the nodal error on the full grid at T."""
    h = tuple(l / n for l, n in zip(LEN, N))
    X = _grid(N, h)[0]
    f = etd.allen_cahn(1 / EPS ** 2, -1 / EPS ** 2)
    src = boundary.boundary_source(N, h, 1.0, f, lambda t: (_wave(t, X), _wave_t(t, X)))
    inner = tuple(slice(1, -1) for _ in N)
    U = etd.make_stepper(N, h, 1.0, T / NT, scheme).run(_wave(0.0, X)[inner].copy(), NT, boundary.with_boundary(f, src))
    E = np.zeros_like(X)
    E[inner] = U - _wave(T, X)[inner]
    return E, h


def _fe_norms(E, N, h):
    """FE L2 and H1 norms of the nodal error (boundary entries 0) with the all-node 1D matrices."""
    AB = [fem.assemble_1d_all_nodes(n, hh) for n, hh in zip(N, h)]
    ME = E
    for a in range(len(N)):
        ME = etd.mode_product(AB[a][0], ME, a)
    KE = 0.0
    for a in range(len(N)):
        T = E
        for b in range(len(N)):
            T = etd.mode_product(AB[b][1] if b == a else AB[b][0], T, b)
        KE = KE + T
    l2sq = float(np.sum(E * ME))
    return math.sqrt(l2sq), math.sqrt(l2sq + float(np.sum(E * KE)))


def _ode_reference(N, T):
    """Example 5.2's semi-discrete system from the global assembly (all nodes, x fastest) with the
    boundary nodes prescribed, integrated by scipy's Radau method to tight tolerances."""
    h = tuple(l / n for l, n in zip(LEN, N))
    M, K, inner = fem.assemble_global_all_nodes(N, h, 1.0)
    X = _grid(N, h)[0].ravel()
    bnd = np.setdiff1d(np.arange(X.size), inner)
    Mii = M[inner][:, inner].toarray()
    Mib, Kii, Kib = M[inner][:, bnd], K[inner][:, inner], K[inner][:, bnd]
    Mall = M[inner]
    fr = lambda u: (u - u ** 3) / EPS ** 2

    def rhs(t, U):
        u = _wave(t, X)
        u[inner] = U
        return np.linalg.solve(Mii, Mall @ fr(u) - Kii @ U - Kib @ u[bnd] - Mib @ _wave_t(t, X[bnd]))

    sol = scipy.integrate.solve_ivp(rhs, (0, T), _wave(0.0, X[inner]), method="Radau", rtol=1e-11, atol=1e-13)
    return sol.y[:, -1], inner, X


@pytest.mark.parametrize("scheme,order", [(1, 1.0), (2, 2.0)])
def test_example52_converges_to_the_semidiscrete_solution(scheme, order):
    """Against a stiff ODE solve of the assembled system (not the oracle's source formula), the error
    at T/4 falls at the scheme's order as tau halves (Theorems 3.1/3.2)."""
    N, T = (16, 4, 4), T_END / 4
    ref, inner, X = _ode_reference(N, T)
    errs = []
    for NT in (16, 32, 64):
        E, h = _example52(N, NT, scheme, T)
        U = (E.ravel() + _wave(T, X))[inner]
        errs.append(np.linalg.norm(U - ref) / np.linalg.norm(ref))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] == pytest.approx(order, abs=0.25), (errs, rates)


def _table4_rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                sc, nt, l2, h1 = line.split()
                rows.append((int(sc), int(nt), float(l2), float(h1)))
    return rows


def test_table4_eife2_l2_errors_are_approached_on_refined_meshes():
    """The printed EIFE2 temporal rows (1024 x 64 x 64) at N_T = 16 and 32: the oracle's L2 errors on
    the 128 x 8 x 8, 256 x 16 x 16 and 512 x 32 x 32 meshes rise monotonically towards them and are
    within 2% and 4% at 512 x 32 x 32 (the GPU test runs the printed mesh)."""
    printed = {nt: l2 for sc, nt, l2, _ in _table4_rows() if sc == 2}
    for NT, tol in ((16, 0.02), (32, 0.04)):
        errs = []
        for N in ((128, 8, 8), (256, 16, 16), (512, 32, 32)):
            E, h = _example52(N, NT, 2)
            errs.append(_fe_norms(E, N, h)[0])
        assert errs[0] < errs[1] < errs[2] < printed[NT] * (1 + tol), (NT, errs)
        assert errs[2] == pytest.approx(printed[NT], rel=tol), (NT, errs)
