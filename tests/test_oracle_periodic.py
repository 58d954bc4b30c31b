"""Pins for the oracle's periodic path and the Flory-Huggins reaction (Section 4, closing remarks on
periodic boundary conditions; Example 5.3 of Section 5.2).

The eigenvalue formulas printed for the periodic case are garbled (an argument (i-1) pi / (2N) and a
missing square); the reading used is theta_i = 2 pi (i-1)/N with
lambda^A_i = (h/6)(6 - 4 sin^2(pi (i-1)/N)) = (h/3)(2 + cos theta_i) and
lambda^B_i = (4/h) sin^2(pi (i-1)/N) = (2/h)(1 - cos theta_i). The references below do not go through
the oracle's eigen path: the printed G^P matrix, a dense matrix-exponential route on tiny grids, the
paper's own DFT route written with the library FFT, the exact decay of a Fourier mode, closed forms
for a constant field, mass conservation, the printed maximum bound gamma ~ 0.9575, and the maximum
bound and energy decay that Example 5.3 reports.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import etd, fem, monitors, spectral
from paper_2209_11922_gb300.inputs import uniform_field

THETA, THETA_C = 0.8, 1.6


def _fh_atanh(u):
    """The Flory-Huggins reaction written independently of the oracle: (theta/2) ln((1-u)/(1+u))
    = -theta artanh(u)."""
    return THETA_C * u - THETA * np.arctanh(u)


# ---------------------------------------------------------------- assembly
@pytest.mark.parametrize("N,h", [(3, 1 / 3), (5, 0.2), (8, 0.125)])
def test_periodic_1d_assembly_matches_printed_matrices(N, h):
    A, B = fem.assemble_1d(N, h, "periodic")
    G = 2 * np.eye(N) - np.roll(np.eye(N), 1, axis=1) - np.roll(np.eye(N), -1, axis=1)   # G^P
    np.testing.assert_allclose(B, G / h, rtol=0, atol=1e-14 / h)
    R = 4 * np.eye(N) + np.roll(np.eye(N), 1, axis=1) + np.roll(np.eye(N), -1, axis=1)
    np.testing.assert_allclose(A, h / 6 * R, rtol=0, atol=1e-15)
    np.testing.assert_allclose(A @ np.ones(N), h * np.ones(N), rtol=1e-14)   # partition of unity


@pytest.mark.parametrize("N,h", [((4, 5), (0.25, 0.2)), ((3, 4, 5), (1 / 3, 0.25, 0.2))])
def test_periodic_global_assembly_matches_kronecker_form(N, h):
    D = 0.7
    M, K = fem.assemble_global(N, h, D, "periodic")
    AB = [fem.assemble_1d(n, hh, "periodic") for n, hh in zip(N, h)]
    d = len(N)

    def kron(mats):   # x fastest: kron(..., A_y, A_x)
        out = np.ones((1, 1))
        for m in reversed(mats):
            out = np.kron(out, m)
        return out

    Mk = kron([AB[a][0] for a in range(d)])
    Kk = sum(D * kron([AB[b][1] if b == a else AB[b][0] for b in range(d)]) for a in range(d))
    np.testing.assert_allclose(M.toarray(), Mk, atol=1e-15)
    np.testing.assert_allclose(K.toarray(), Kk, atol=1e-12)


# ---------------------------------------------------------------- eigenvalues
@pytest.mark.parametrize("N,h", [(4, 0.25), (7, 1 / 7), (16, 1 / 16), (12, 0.3)])
def test_periodic_eigenvalues_match_corrected_closed_form(N, h):
    e = spectral.axis_eigen(N, h, "periodic")
    i = np.arange(1, N + 1)
    s2 = np.sin(np.pi * (i - 1) / N) ** 2
    lamA = h / 6 * (6 - 4 * s2)
    lamB = 4 / h * s2
    order = np.argsort(e.lamA)
    np.testing.assert_allclose(np.sort(e.lamA), np.sort(lamA), rtol=1e-13)
    np.testing.assert_allclose(np.sort(e.lamB), np.sort(lamB), atol=1e-12 / h)
    assert e.offdiag < 1e-12 / h
    # mu pairs with lambda^A: the largest mass eigenvalue (mode 0) has rate 0
    th = 2 * np.pi * (i - 1) / N
    mu = 6 * (1 - np.cos(th)) / (h * h * (2 + np.cos(th)))
    np.testing.assert_allclose(np.sort(e.mu), np.sort(mu), atol=1e-10 / h ** 2)
    assert abs(e.mu[order[-1]]) < 1e-10 / h ** 2


def test_printed_periodic_eigenvalues_are_not_eigenvalues():
    """The printed lambda^A with sin((i-1) pi / (2N)) and no square is not the spectrum."""
    N, h = 8, 0.125
    e = spectral.axis_eigen(N, h, "periodic")
    i = np.arange(1, N + 1)
    printed = h / 6 * (6 - 4 * np.sin((i - 1) * np.pi / (2 * N)))
    assert np.abs(np.sort(printed) - np.sort(e.lamA)).max() > 0.1 * h


# ---------------------------------------------------------------- dense expm path (tiny grids)
def _dense_step(U, L, tau, scheme, c2, f, t):
    from test_oracle_scheme import _dense_step as ds
    return ds(U, L, tau, scheme, c2, f, t)


@pytest.mark.parametrize("N,h", [((4, 5), (0.25, 0.2)), ((3, 4, 3), (1 / 3, 0.25, 1 / 3))])
@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("react", ["allen_cahn", "flory_huggins"])
def test_periodic_eigen_path_matches_dense_expm(N, h, scheme, react):
    D, tau, nsteps, c2 = 0.05, 0.03, 3, 0.5
    M, K = fem.assemble_global(N, h, D, "periodic")
    L = np.linalg.solve(M.toarray(), K.toarray())
    U0 = uniform_field(tuple(reversed(N)), -0.9, 0.9, seed=17)
    if react == "allen_cahn":
        fo, fd = etd.allen_cahn(1.0, -1.0), (lambda t, x: x - x ** 3)
    else:
        fo, fd = etd.flory_huggins(THETA, THETA_C), (lambda t, x: _fh_atanh(x))
    u = U0.ravel().copy()
    for n in range(nsteps):
        u = _dense_step(u, L, tau, scheme, c2, fd, n * tau)
    got = etd.make_stepper(N, h, D, tau, scheme, c2, "periodic").run(U0, nsteps, fo)
    np.testing.assert_allclose(got.ravel(), u, rtol=1e-12, atol=1e-13)


# ---------------------------------------------------------------- the paper's DFT route
def _phi12(z):
    """phi_1, phi_2 of real z <= 0 in closed form, with Taylor series near 0."""
    z = np.asarray(z, dtype=np.float64)
    small = np.abs(z) < 1e-3
    zs = np.where(small, 1.0, z)
    p1 = np.where(small, 1 + z / 2 + z * z / 6 + z ** 3 / 24, np.expm1(zs) / zs)
    p2 = np.where(small, 0.5 + z / 6 + z * z / 24 + z ** 3 / 120, (np.expm1(zs) - zs) / (zs * zs))
    return p1, p2


def _dft_step(U, N, h, D, tau, scheme, f, c2=0.5):
    """One EIFE step by a DFT along each axis and the closed-form rates mu(2 pi k / N)."""
    mus = []
    for n, hh in zip(N, h):
        th = 2 * np.pi * np.arange(n) / n
        mus.append(6 * (1 - np.cos(th)) / (hh * hh * (2 + np.cos(th))))
    H = np.zeros(U.shape)
    for a, m in enumerate(mus):
        shape = [1] * U.ndim
        shape[U.ndim - 1 - a] = len(m)
        H = H + D * m.reshape(shape)
    z = -tau * H
    E = np.exp(z)
    p1, p2 = _phi12(z)
    Ec = np.exp(c2 * z)
    p1c, _ = _phi12(c2 * z)
    F, iF = np.fft.fftn, lambda X: np.real(np.fft.ifftn(X))
    Ut, G1 = F(U), F(f(0.0, U))
    if scheme == 1:
        return iF(E * Ut + tau * p1 * G1)
    U2 = iF(Ec * Ut + c2 * tau * p1c * G1)
    G2 = F(f(0.0, U2))
    return iF(E * Ut + tau * (p1 - p2 / c2) * G1 + tau * (p2 / c2) * G2)


@pytest.mark.parametrize("N", [(16, 12), (8, 6, 10)])
@pytest.mark.parametrize("scheme", [1, 2])
def test_periodic_step_matches_the_dft_route(N, scheme):
    h = tuple(1.0 / n for n in N)
    D, tau = 1e-2, 0.02
    U = uniform_field(tuple(reversed(N)), -0.9, 0.9, seed=23)
    st = etd.make_stepper(N, h, D, tau, scheme, 0.5, "periodic")
    f = etd.flory_huggins(THETA, THETA_C)
    ref = U.copy()
    got = U.copy()
    for _ in range(3):
        ref = _dft_step(ref, N, h, D, tau, scheme, lambda t, x: _fh_atanh(x))
        got = st.step(got, 0.0, f)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


# ---------------------------------------------------------------- closed forms and invariants
@pytest.mark.parametrize("scheme", [1, 2])
def test_fourier_mode_decays_exactly_when_f_is_zero(scheme):
    N, D, tau, n = (24, 16), 3e-3, 0.05, 7
    h = tuple(1.0 / m for m in N)
    p, q = 5, 3
    x = np.arange(N[0]) * h[0]
    y = np.arange(N[1]) * h[1]
    U0 = np.outer(np.sin(2 * np.pi * q * y + 0.3), np.cos(2 * np.pi * p * x))
    mu = lambda k, m, hh: 6 * (1 - np.cos(2 * np.pi * k / m)) / (hh * hh * (2 + np.cos(2 * np.pi * k / m)))
    ref = math.exp(-n * tau * D * (mu(p, N[0], h[0]) + mu(q, N[1], h[1]))) * U0
    got = etd.run(U0, N, h, D, tau, n, scheme, flin=0.0, fcub=0.0, bc="periodic")
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("scheme", [1, 2])
def test_constant_field_follows_the_scalar_scheme(scheme):
    """A constant field has no diffusion (B 1 = 0), so it follows the scheme with zero linear part:
    EIFE1 is forward Euler and EIFE2 with c2 = 1/2 is the midpoint rule."""
    N, h, D, tau, c = (6, 5, 4), (1 / 6, 0.2, 0.25), 0.1, 0.05, 0.37
    U = np.full((4, 5, 6), c)
    st = etd.make_stepper(N, h, D, tau, scheme, 0.5, "periodic")
    f = etd.flory_huggins(THETA, THETA_C)
    for _ in range(5):
        U = st.step(U, 0.0, f)
        c = c + tau * _fh_atanh(c) if scheme == 1 else c + tau * _fh_atanh(c + 0.5 * tau * _fh_atanh(c))
        np.testing.assert_allclose(U, c, rtol=1e-13)


def test_mass_is_conserved_without_reaction():
    N, h = (8, 12, 10), (0.125, 1 / 12, 0.1)
    U = uniform_field((10, 12, 8), -0.9, 0.9, seed=3)
    m0 = monitors.monitors(U, N, h, 1.0, "periodic")["mass"]
    V = etd.run(U, N, h, 0.02, 0.05, 6, 2, flin=0.0, fcub=0.0, bc="periodic")
    m1 = monitors.monitors(V, N, h, 1.0, "periodic")["mass"]
    assert m1 == pytest.approx(m0, rel=1e-12, abs=1e-14)
    assert m0 == pytest.approx(np.prod(h) * U.sum(), rel=1e-13)   # A 1 = h 1 per axis


def test_flory_huggins_max_bound_matches_printed_gamma():
    """Example 5.3 prints gamma ~ 0.9575 for theta = 0.8, theta_c = 1.6."""
    g = monitors.fh_max_bound(THETA, THETA_C)
    assert round(g, 4) == 0.9575
    assert abs(_fh_atanh(g)) < 1e-12


def test_reaction_forms_agree():
    u = np.linspace(-0.95, 0.95, 41)
    a = etd.flory_huggins(THETA, THETA_C)(0.0, u)
    b = etd.reaction(THETA_C, 0.0, -THETA)(0.0, u)
    np.testing.assert_allclose(a, _fh_atanh(u), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(b, _fh_atanh(u), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("N,h", [((6, 5), (1 / 6, 0.2)), ((4, 5, 3), (0.25, 0.2, 1 / 3))])
def test_periodic_monitors_match_global_assembly(N, h):
    D = 1e-2
    U = uniform_field(tuple(reversed(N)), -0.9, 0.9, seed=4)
    M, K = fem.assemble_global(N, h, D, "periodic")
    u = U.ravel()
    m = monitors.monitors(U, N, h, D, "periodic", flory_huggins=(THETA, THETA_C))
    assert m["mass"] == pytest.approx(float(np.ones_like(u) @ (M @ u)), rel=1e-13)
    quad = 0.5 * float(u @ (K @ u))
    # the potential's derivative is -f: check it on constant fields (no gradient term)
    c, d = 0.41, 1e-5
    e = lambda v: monitors.monitors(np.full(U.shape, v), N, h, D, "periodic", (THETA, THETA_C))["energy"]
    dE = (e(c + d) - e(c - d)) / (2 * d) / (np.prod(h) * u.size)
    assert dE == pytest.approx(-_fh_atanh(c), rel=1e-7)
    pot = m["energy"] - quad
    assert e(0.0) == pytest.approx(0.0, abs=1e-15)
    assert pot == pytest.approx(np.prod(h) * np.sum(
        THETA * (u * np.arctanh(u) + 0.5 * np.log1p(-u * u)) - 0.5 * THETA_C * u * u), rel=1e-12)


def test_example53_keeps_the_max_bound_and_decays_the_energy():
    """Example 5.3's parameters on a 16^3 mesh (same eps, theta, theta_c, tau and initial law):
    max|u| stays below gamma and the discrete energy does not increase (Section 5.2)."""
    N = (16, 16, 16)
    h = (1 / 16,) * 3
    D, tau = 1e-4, 20.0 / 2048
    U = uniform_field((16, 16, 16), -0.9, 0.9, seed=11)
    st = etd.make_stepper(N, h, D, tau, 2, 0.5, "periodic")
    f = etd.flory_huggins(THETA, THETA_C)
    g = monitors.fh_max_bound(THETA, THETA_C)
    E = monitors.monitors(U, N, h, D, "periodic", (THETA, THETA_C))["energy"]
    for _ in range(40):
        U = st.step(U, 0.0, f)
        m = monitors.monitors(U, N, h, D, "periodic", (THETA, THETA_C))
        assert m["maxabs"] <= g
        assert m["energy"] <= E + 1e-14
        E = m["energy"]
    assert m["maxabs"] > 0.9 * g   # the field has separated into the two phases


# ---------------------------------------------------------------- the Hartley transform (kernel-level oracle)
@pytest.mark.parametrize("N", [4, 6, 16, 48])
def test_hartley_matrix_is_the_real_form_of_the_dft(N):
    from oracle import transforms
    H = transforms.hartley_matrix(N)
    F = np.fft.fft(np.eye(N), axis=0)          # F_jk = exp(-2 pi i j k / N)
    np.testing.assert_allclose(H, (F.real - F.imag) / np.sqrt(N), atol=1e-14)
    np.testing.assert_allclose(H @ H, np.eye(N), atol=1e-13)
    A, B = fem.assemble_1d(N, 1.0 / N, "periodic")
    th = 2 * np.pi * np.arange(N) / N
    np.testing.assert_allclose(H @ A @ H, np.diag((2 + np.cos(th)) / (3 * N)), atol=1e-14)
    np.testing.assert_allclose(H @ B @ H, np.diag(2 * N * (1 - np.cos(th))), atol=1e-10)


def test_double_well_energy_is_the_allen_cahn_potential():
    """The monitors' default potential is pinned by the reaction it belongs to: on constant periodic
    fields (no gradient term) dE/du = -(u - u^3) per unit volume, and E vanishes in the wells u = +-1."""
    N, h = (6, 5, 4), (1 / 6, 0.2, 0.25)
    vol = np.prod(h) * np.prod(N)
    e = lambda v: monitors.monitors(np.full((4, 5, 6), v), N, h, 0.3, "periodic")["energy"]
    for c in (-0.7, 0.2, 0.55, 1.3):
        d = 1e-5
        assert (e(c + d) - e(c - d)) / (2 * d) / vol == pytest.approx(-(c - c ** 3), rel=1e-7, abs=1e-10)
    assert e(1.0) == pytest.approx(0.0, abs=1e-15) and e(-1.0) == pytest.approx(0.0, abs=1e-15)
