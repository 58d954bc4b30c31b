"""Pins for the oracle's assembly and eigen-decomposition (Sections 2.1 and 4).

Each test checks the oracle against something other than itself: quadrature of explicit basis
functions, the matrices printed with eq. (4.1), and the closed-form eigenpairs of tridiagonal
Toeplitz matrices.
"""
import itertools

import numpy as np
import pytest

from oracle import fem, spectral


def _hat_1d(h, which, x):
    """Linear shape function on [0, h]: node 0 -> 1 - x/h, node 1 -> x/h; and its derivative."""
    if which == 0:
        return 1.0 - x / h, -np.ones_like(x) / h
    return x / h, np.ones_like(x) / h


@pytest.mark.parametrize("h", [0.1, 0.37, 2.0 / 2048])
def test_element_matrices_1d_by_quadrature(h):
    gx, gw = np.polynomial.legendre.leggauss(3)
    x, w = 0.5 * h * (gx + 1), 0.5 * h * gw
    me, ke = fem.element_mass_1d(h), fem.element_stiffness_1d(h)
    for a in range(2):
        for b in range(2):
            fa, da = _hat_1d(h, a, x)
            fb, db = _hat_1d(h, b, x)
            assert me[a, b] == pytest.approx(np.sum(w * fa * fb), rel=1e-14)
            assert ke[a, b] == pytest.approx(np.sum(w * da * db), rel=1e-14)


@pytest.mark.parametrize("h", [(0.3, 0.7), (0.25, 0.5, 0.125)])
def test_element_matrices_nd_by_quadrature(h):
    """Tensor Gauss quadrature of the explicit Q1 basis functions and their gradients."""
    d, D = len(h), 0.37
    Me, Ke = fem.element_matrices_nd(h, D)
    gx, gw = np.polynomial.legendre.leggauss(3)
    pts = [0.5 * ha * (gx + 1) for ha in h]
    wts = [0.5 * ha * gw for ha in h]
    locs = [tuple((n >> a) & 1 for a in range(d)) for n in range(2 ** d)]
    for p, ip in enumerate(locs):
        for q, iq in enumerate(locs):
            m = k = 0.0
            for qi in itertools.product(range(3), repeat=d):
                wq = np.prod([wts[a][qi[a]] for a in range(d)])
                vp = [_hat_1d(h[a], ip[a], pts[a][qi[a]]) for a in range(d)]
                vq = [_hat_1d(h[a], iq[a], pts[a][qi[a]]) for a in range(d)]
                fp = np.prod([v[0] for v in vp])
                fq = np.prod([v[0] for v in vq])
                gp = [vp[a][1] * np.prod([vp[b][0] for b in range(d) if b != a]) for a in range(d)]
                gq = [vq[a][1] * np.prod([vq[b][0] for b in range(d) if b != a]) for a in range(d)]
                m += wq * fp * fq
                k += wq * D * float(np.dot(gp, gq))
            assert Me[p, q] == pytest.approx(m, rel=1e-13, abs=1e-16)
            assert Ke[p, q] == pytest.approx(k, rel=1e-13, abs=1e-14)


@pytest.mark.parametrize("N,h", [(2, 0.5), (7, 0.2), (64, 1 / 64)])
def test_assembled_1d_matches_eq41(N, h):
    """A = (h/6) R_{N-1}, B = (1/h) G^D_{N-1} as printed with eq. (4.1)."""
    A, B = fem.assemble_1d(N, h)
    n = N - 1
    R = 4 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
    G = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    np.testing.assert_allclose(A, h / 6 * R, rtol=1e-15, atol=1e-16)
    np.testing.assert_allclose(B, G / h, rtol=1e-15, atol=1e-16)


@pytest.mark.parametrize("N,h", [((5, 7), (0.2, 1 / 7.0)), ((3, 4, 5), (0.5, 0.25, 0.3))])
def test_global_assembly_matches_kronecker_form(N, h):
    """Global Q1 M and K (element by element) against eq. (4.1), by random matvecs."""
    D = 0.013
    M, K = fem.assemble_global(N, h, D)
    AB = [fem.assemble_1d(n, hh) for n, hh in zip(N, h)]
    d = len(N)

    def kron_x_fastest(mats):  # x is the fastest index -> kron(z, y, x)
        out = np.ones((1, 1))
        for m in reversed(mats):
            out = np.kron(out, m)
        return out

    Mk = kron_x_fastest([AB[a][0] for a in range(d)])
    Kk = sum(D * kron_x_fastest([AB[b][1] if b == a else AB[b][0] for b in range(d)]) for a in range(d))
    rng = np.random.default_rng(1)
    for _ in range(4):
        v = rng.standard_normal(M.shape[0])
        np.testing.assert_allclose(M @ v, Mk @ v, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(K @ v, Kk @ v, rtol=1e-13, atol=1e-13)


def _closed_form(N, h):
    i = np.arange(1, N)
    th = i * np.pi / N
    lamA = h / 3 * (2 + np.cos(th))            # (h/6)(6 - 4 sin^2(theta/2))
    lamB = 4 / h * np.sin(th / 2) ** 2
    mu = 6 / h ** 2 * (1 - np.cos(th)) / (2 + np.cos(th))
    S = np.sqrt(2.0 / N) * np.sin(np.outer(i, i) * np.pi / N)
    return lamA, lamB, mu, S


@pytest.mark.parametrize("N,h", [(4, 0.25), (16, 1 / 16), (63, 0.01), (256, 1 / 256)])
def test_eigenpairs_match_corrected_closed_form(N, h):
    """Section 4's simultaneous diagonalisation, with the squared sine in lambda^A and the
    orthonormal sine matrix (Section 4 prints lambda^A without the square and calls the unscaled
    sine matrix orthogonal)."""
    e = spectral.axis_eigen(N, h)
    lamA, lamB, mu, S = _closed_form(N, h)
    assert e.offdiag <= 1e-12 * np.max(np.abs(lamB))
    # the oracle's eigenvalues and the closed form, both sorted by mu
    o = np.argsort(e.mu)
    c = np.argsort(mu)
    np.testing.assert_allclose(e.mu[o], mu[c], rtol=1e-11)
    np.testing.assert_allclose(e.lamA[o], lamA[c], rtol=1e-12)
    np.testing.assert_allclose(e.lamB[o], lamB[c], rtol=1e-10, atol=1e-12 * lamB.max())
    # eigenvectors equal the orthonormal sine columns up to sign
    for k in range(N - 1):
        col = e.P[:, o[k]]
        ref = S[:, c[k]]
        assert min(np.abs(col - ref).max(), np.abs(col + ref).max()) < 1e-10
    np.testing.assert_allclose(S @ S, np.eye(N - 1), atol=1e-13)


def test_printed_lambdaA_without_square_is_not_an_eigenvalue():
    """The formula as printed in Section 4, (h/6)(6 - 4 sin(i pi / 2N)), does not match A's spectrum."""
    N, h = 16, 1 / 16
    e = spectral.axis_eigen(N, h)
    i = np.arange(1, N)
    printed = h / 6 * (6 - 4 * np.sin(i * np.pi / (2 * N)))
    assert np.max(np.abs(np.sort(printed) - np.sort(e.lamA))) > 1e-3 * h


def test_mode_rates_sum_per_axis():
    mus = [np.array([1.0, 2.0, 3.0]), np.array([10.0, 20.0])]
    H = spectral.mode_rates(mus, 0.5)
    assert H.shape == (2, 3)  # storage order (y, x)
    np.testing.assert_allclose(H, 0.5 * (np.array([[10.0], [20.0]]) + np.array([[1.0, 2.0, 3.0]])))


@pytest.mark.parametrize("N", [4, 6, 33, 96])
def test_sine_matrix_is_the_numerical_eigenbasis(N):
    """oracle.transforms.sine_matrix diagonalises the assembled A and B and is an involution."""
    from oracle import transforms
    S = transforms.sine_matrix(N)
    A, B = fem.assemble_1d(N, 1.0 / N)
    for M in (A, B):
        D = S @ M @ S
        assert np.abs(D - np.diag(np.diag(D))).max() < 1e-12 * np.abs(M).max()
    np.testing.assert_allclose(S @ S, np.eye(N - 1), atol=1e-13)


@pytest.mark.parametrize("N,h", [((6, 5), (1 / 6, 0.2)), ((4, 5, 3), (0.25, 0.2, 1 / 3))])
def test_monitors_match_global_assembly(N, h):
    """mass = 1^T M U and the quadratic energy term 1/2 U^T K U against the globally assembled M, K."""
    from oracle import monitors
    from paper_2209_11922_gb300.inputs import uniform_field
    D = 0.3
    U = uniform_field(tuple(n - 1 for n in reversed(N)), -1, 1, seed=2)
    M, K = fem.assemble_global(N, h, D)
    u = U.ravel()
    m = monitors.monitors(U, N, h, D)
    assert m["mass"] == pytest.approx(float(np.ones_like(u) @ (M @ u)), rel=1e-13)
    pot = np.prod(h) * 0.25 * np.sum((u * u - 1) ** 2)
    assert m["energy"] == pytest.approx(0.5 * float(u @ (K @ u)) + pot, rel=1e-13)
    assert m["maxabs"] == pytest.approx(np.abs(u).max()) and m["nonfinite"] == 0
