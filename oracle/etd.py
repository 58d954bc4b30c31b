"""EIFE1 and EIFE2 time steps in the spectral form of Section 4.

With U~ = S_x^T (x) S_y^T (x) S_z^T (x) U (tensor mode products of Section 4, S orthonormal),
eq. (4.3) reads dU~/dt + H (.) U~ = S^T F(t, S U~)  (nodal reading F = M f(U), which cancels the
tensor H^ of Section 4), and the EIFE schemes are applied mode by mode:

EIFE1, eq. (2.13):
    U~^{n+1} = e^{-tau H} U~^n + tau phi_1(-tau H) G~_1,           G_1 = f(t_n, U^n)
EIFE2, eq. (2.14), c_1 = 0, c_2 in (0, 1]:
    U~_2     = e^{-c2 tau H} U~^n + c2 tau phi_1(-c2 tau H) G~_1
    G_2      = f(t_n + c2 tau, S U~_2)
    U~^{n+1} = e^{-tau H} U~^n + tau [(phi_1 - phi_2/c2)(-tau H) G~_1 + (phi_2/c2)(-tau H) G~_2]

Every step starts from the physical nodal field and returns it, applying the transforms as dense
products along each axis (no fusion, no FFT). The periodic case (Section 4, closing remarks) is the
same scheme on the circulant matrices' orthonormal eigenbasis (Section 4 applies it by a DFT per
axis; here the basis is numerical, and the FFT form is a pin). Parity: pinned (dense
matrix-exponential path on tiny grids, both boundary conditions; exact decay of a sine or Fourier
mode with f = 0; per-mode closed forms for linear f; a constant periodic field following the scalar
scheme with zero linear part; the temporal orders of Theorems 3.1/3.2; the EIFE rows of Table 2;
the maximum bound and energy decay of Example 5.3).
"""
from __future__ import annotations

from typing import Callable, Sequence

import numpy as np

from .phi import phi
from .spectral import axis_eigen, mode_rates

Reaction = Callable[[float, np.ndarray], np.ndarray]


def mode_product(M: np.ndarray, U: np.ndarray, axis: int) -> np.ndarray:
    """(M (x)_a U): contract M's second index with paper axis ``axis`` (0 = x, 1 = y, 2 = z).

    Storage order is (z, y, x), so paper axis a is array axis ndim-1-a.
    """
    ax = U.ndim - 1 - axis
    return np.moveaxis(np.tensordot(M, U, axes=([1], [ax])), 0, ax)


def forward(U: np.ndarray, Ps: Sequence[np.ndarray]) -> np.ndarray:
    """U~ = P_x^T (x) P_y^T (x) P_z^T (x) U."""
    for a, P in enumerate(Ps):
        U = mode_product(P.T, U, a)
    return U


def inverse(Ut: np.ndarray, Ps: Sequence[np.ndarray]) -> np.ndarray:
    """U = P_x (x) P_y (x) P_z (x) U~."""
    for a, P in enumerate(Ps):
        Ut = mode_product(P, Ut, a)
    return Ut


def allen_cahn(flin: float = 1.0, fcub: float = -1.0) -> Reaction:
    """f(t, u) = flin * u + fcub * u^3 on nodal values (Allen-Cahn: flin = 1, fcub = -1)."""
    def f(t, u):
        return flin * u + fcub * u * u * u
    return f


def flory_huggins(theta: float, theta_c: float) -> Reaction:
    """f(u) = (theta/2) ln((1 - u)/(1 + u)) + theta_c u, the Flory-Huggins reaction of Example 5.3
    (Section 5.2), on nodal values; defined for |u| < 1."""
    def f(t, u):
        return 0.5 * theta * np.log((1.0 - u) / (1.0 + u)) + theta_c * u
    return f


def reaction(flin: float = 1.0, fcub: float = -1.0, flog: float = 0.0) -> Reaction:
    """f(u) = flin u + fcub u^3 + flog * (1/2) ln((1 + u)/(1 - u)): the Allen-Cahn family plus a
    logarithmic term (Flory-Huggins: flin = theta_c, fcub = 0, flog = -theta)."""
    def f(t, u):
        out = flin * u + fcub * u * u * u
        if flog != 0.0:
            out = out + flog * 0.5 * np.log((1.0 + u) / (1.0 - u))
        return out
    return f


class Stepper:
    """EIFE1/EIFE2 on given per-axis orthonormal eigenvector matrices and per-mode rates H."""

    def __init__(self, Ps: Sequence[np.ndarray], H: np.ndarray, tau: float, scheme: int,
                 c2: float = 0.5):
        if scheme not in (1, 2):
            raise ValueError("scheme must be 1 (EIFE1) or 2 (EIFE2)")
        if not (0.0 < c2 <= 1.0):
            raise ValueError("c2 must lie in (0, 1]")
        self.Ps, self.tau, self.scheme, self.c2 = list(Ps), float(tau), scheme, float(c2)
        z = -tau * H
        self.E = phi(0, z)
        self.phi1 = phi(1, z)
        self.phi2 = phi(2, z)
        self.Ec = phi(0, c2 * z)
        self.phi1c = phi(1, c2 * z)

    def step(self, U: np.ndarray, t: float, f: Reaction) -> np.ndarray:
        tau, c2 = self.tau, self.c2
        Ut = forward(U, self.Ps)
        G1t = forward(f(t, U), self.Ps)
        if self.scheme == 1:
            return inverse(self.E * Ut + tau * self.phi1 * G1t, self.Ps)
        U2t = self.Ec * Ut + c2 * tau * self.phi1c * G1t
        G2t = forward(f(t + c2 * tau, inverse(U2t, self.Ps)), self.Ps)
        Unt = (self.E * Ut + tau * (self.phi1 - self.phi2 / c2) * G1t
               + tau * (self.phi2 / c2) * G2t)
        return inverse(Unt, self.Ps)

    def run(self, U: np.ndarray, nsteps: int, f: Reaction, t0: float = 0.0) -> np.ndarray:
        for n in range(nsteps):
            U = self.step(U, t0 + n * self.tau, f)
        return U


def make_stepper(N: Sequence[int], h: Sequence[float], D: float, tau: float, scheme: int,
                 c2: float = 0.5, bc: str = "dirichlet") -> Stepper:
    """Assemble the 1D matrices per axis (``bc`` 'dirichlet' or 'periodic'), diagonalise them, and
    build the stepper. Periodic fields have N_a nodes per axis, Dirichlet fields N_a - 1."""
    eig = [axis_eigen(int(n), float(hh), bc) for n, hh in zip(N, h)]
    H = mode_rates([e.mu for e in eig], D)
    return Stepper([e.P for e in eig], H, tau, scheme, c2)


def run(u0: np.ndarray, N: Sequence[int], h: Sequence[float], D: float, tau: float, nsteps: int,
        scheme: int = 2, c2: float = 0.5, flin: float = 1.0, fcub: float = -1.0, bc: str = "dirichlet",
        flog: float = 0.0) -> np.ndarray:
    """``nsteps`` EIFE steps of u_t = D Lap u + f(u), f = flin u + fcub u^3 [+ flog atanh u], from
    nodal ``u0`` (float64)."""
    st = make_stepper(N, h, D, tau, scheme, c2, bc)
    f = allen_cahn(flin, fcub) if flog == 0.0 else reaction(flin, fcub, flog)
    return st.run(np.asarray(u0, dtype=np.float64), nsteps, f)
