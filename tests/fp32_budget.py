"""Error budget of an FP32 implementation of the EIFE1/EIFE2 step (eqs. (2.13)/(2.14) in the
spectral form of Section 4), measured on the CPU.

``run`` takes the scheme of the CPU oracle with three independent switches: the state and the
reaction kept in float32 (``state32``), the per-mode coefficients computed in FP64 from the
closed-form eigenvalues and rounded once to float32 (``coef32``), and every transform computed in
float32 by the library FFT's DST-I (``dst32``; otherwise the transforms run in FP64 on the same
values). Each switch alone shows what that part of an FP32 pipeline costs against the FP64 oracle.
Test infrastructure only.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft


def mu(N: int, h: float) -> np.ndarray:
    """Closed-form 1D rates (6/h^2)(1 - cos t)/(2 + cos t), t = i pi / N, i = 1..N-1 (Section 4 with
    the squared sine of lambda^A restored)."""
    t = np.arange(1, N) * np.pi / N
    return 6.0 / (h * h) * (1.0 - np.cos(t)) / (2.0 + np.cos(t))


def phi12(z: np.ndarray):
    """phi_1(z), phi_2(z) in FP64 for z <= 0: series below |z| = 0.5, closed form above."""
    z = np.asarray(z, dtype=np.float64)
    p1 = np.empty_like(z)
    p2 = np.empty_like(z)
    s = np.abs(z) < 0.5
    zs = z[s]
    # sum_m z^m/(m+1)!, sum_m z^m/(m+2)! to 20 terms (|z| < 0.5: truncation < 1e-25)
    t1 = np.zeros_like(zs)
    t2 = np.zeros_like(zs)
    f1, f2 = 1.0, 0.5
    zp = np.ones_like(zs)
    for m in range(20):
        t1 += zp * f1
        t2 += zp * f2
        zp = zp * zs
        f1 /= (m + 2)
        f2 /= (m + 3)
    p1[s], p2[s] = t1, t2
    zl = z[~s]
    e = np.expm1(zl)
    p1[~s] = e / zl
    p2[~s] = (e - zl) / (zl * zl)
    return p1, p2


def run(u0, N, h, D, tau, nsteps, scheme=2, c2=0.5, flin=1.0, fcub=-1.0,
        state32=True, coef32=True, dst32=True):
    """nsteps EIFE steps of u_t = D Lap u + flin u + fcub u^3 (see the module docstring)."""
    mus = [mu(int(n), float(hh)) for n, hh in zip(N, h)]
    nd = len(mus)
    H = np.zeros([len(m) for m in reversed(mus)])
    for a, m in enumerate(mus):
        shp = [1] * nd
        shp[nd - 1 - a] = len(m)
        H = H + D * m.reshape(shp)
    z = -tau * H
    p1, p2 = phi12(z)
    cdt = np.float32 if coef32 else np.float64
    sdt = np.float32 if state32 else np.float64
    tdt = np.float32 if dst32 else np.float64
    C = lambda a: np.asarray(a, dtype=cdt)
    S = lambda a: np.asarray(a, dtype=sdt)
    if scheme == 1:
        cE, cG = C(np.exp(z)), C(tau * p1)
    else:
        p1c, _ = phi12(c2 * z)
        cEc, cG1c = C(np.exp(c2 * z)), C(c2 * tau * p1c)
        cE, cA, cB = C(np.exp(z)), C(tau * (p1 - p2 / c2)), C(tau * p2 / c2)
    fl, fc = sdt(flin), sdt(fcub)
    f = lambda u: S(u * (fl + fc * u * u))

    def tr(U):   # orthonormal DST-I along every axis (its own inverse)
        V = np.asarray(U, dtype=tdt)
        for ax in range(nd):
            V = sfft.dst(V, type=1, norm="ortho", axis=ax)
        return S(V)

    U = S(u0)
    for _ in range(nsteps):
        Ut, G1 = tr(U), tr(f(U))
        if scheme == 1:
            U = tr(S(cE * Ut + cG * G1))
        else:
            G2 = tr(f(tr(S(cEc * Ut + cG1c * G1))))
            U = tr(S(cE * Ut + cA * G1 + cB * G2))
    return np.asarray(U, dtype=np.float64)
