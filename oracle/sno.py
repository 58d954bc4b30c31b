"""Spectral neural operator (SNO): the learned coarse propagator of the Parareal loop - plain FP64
forward pass, its gradient written out by the chain rule, the Adam update, and the Parareal
iteration itself. TEST INFRASTRUCTURE ONLY (see the package docstring).

The operator maps a nodal field u (interior nodes of an N x N mesh, shape (B, N-1, N-1)) and the
diffusion coefficient D to a prediction of the field a fixed number of ETDRK2 steps later. Its
spectral layers use the orthonormal sine basis of Section 4 truncated to the lowest M modes per
axis, S_M[p][j] = sqrt(2/N) sin((p+1)(j+1) pi / N), p < M, j < N-1:

    a      = (ln D - ln 1e-3) / ln 100                         (input feature, ~[-1/2, 1/2])
    h_0[c] = Wl[c,0] u + Wl[c,1] a + bl[c]                      (lift, c < C)
    layer l = 0..L-1:
      hh[c]    = S_M (bf(h_l[c]) bf(S_M)^T)                     (M x M modes; the inner product bf16)
      gh[o]    = sum_c bf(Wm[l,p,q,o,c]) bf(hh[c,p,q])          (per-mode channel mix, bf16 operands)
      z_l[o]   = bf(S_M)^T bf(gh[o] S_M) + sum_c bf(Wp[l,o,c]) bf(h_l[c]) + bp[l,o]
      h_{l+1}  = gelu(z_l),  gelu(z) = z/2 (1 + erf(z / sqrt 2))
    u_hat  = u + sum_c Wq[c] h_L[c] + bq                        (projection onto the increment)

bf(x) rounds to bfloat16 (round to nearest, ties to even) after rounding to float32, the precision
the CUDA path rounds from. The bf16 operands are those of the contractions that run on bf16 tensor cores
(the channel-mixing layers, and the two contractions over the mesh of the truncated transforms) and of
the per-mode mix. Loss: mean squared error over all nodes of the batch. The gradient treats bf as the
identity (straight-through), so the mix gradients use the rounded operands.
Parity: pinned by central finite differences of the loss (tests/test_oracle_sno.py), by the
transform (S_M equals the leading rows of the oracle's sine matrix), and by gelu's closed forms.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from math import erf, log, pi, sqrt

import numpy as np

from .transforms import sine_matrix

_erf = np.vectorize(erf, otypes=[np.float64])


def feature(D) -> np.ndarray:
    """Input feature of the diffusion coefficient: (ln D - ln 1e-3) / ln 100."""
    return (np.log(np.asarray(D, dtype=np.float64)) - log(1e-3)) / log(100.0)


def bf16(x) -> np.ndarray:
    """Round to float32, then to bfloat16 (nearest, ties to even); returned as float64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def mode_matrix(N: int, M: int) -> np.ndarray:
    """S_M: the first M rows of the orthonormal sine matrix of an axis with N intervals."""
    return sine_matrix(N)[:M]


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / sqrt(2.0)))


def gelu_grad(z):
    """d gelu / dz = Phi(z) + z phi(z) (standard normal CDF and density)."""
    return 0.5 * (1.0 + _erf(z / sqrt(2.0))) + z * np.exp(-0.5 * z * z) / sqrt(2.0 * pi)


@dataclass
class Params:
    Wl: np.ndarray   # (C, 2)
    bl: np.ndarray   # (C,)
    Wm: np.ndarray   # (L, M, M, C, C)  [l, p, q, o, c]
    Wp: np.ndarray   # (L, C, C)        [l, o, c]
    bp: np.ndarray   # (L, C)
    Wq: np.ndarray   # (C,)
    bq: np.ndarray   # ()

    NAMES = ("Wl", "bl", "Wm", "Wp", "bp", "Wq", "bq")

    def arrays(self):
        return [getattr(self, n) for n in self.NAMES]

    def copy(self) -> "Params":
        return Params(*[np.array(a, dtype=np.float64, copy=True) for a in self.arrays()])


def zeros_like(p: Params) -> Params:
    return Params(*[np.zeros_like(a) for a in p.arrays()])


@dataclass
class Cache:
    u: np.ndarray
    a: np.ndarray
    h: list = field(default_factory=list)    # h_0 .. h_L, each (B, C, n, n)
    z: list = field(default_factory=list)    # z_0 .. z_{L-1}
    hh: list = field(default_factory=list)   # bf-rounded modes of h_l, (B, C, M, M)


def forward(P: Params, u: np.ndarray, D, N: int, rounding: bool = True) -> tuple:
    """u_hat for fields u (B, N-1, N-1) and coefficients D (B,); returns (u_hat, cache).
    rounding=False replaces bf by the identity (used by the finite-difference pin of backward)."""
    bf = bf16 if rounding else (lambda x: np.asarray(x, dtype=np.float64))
    u = np.asarray(u, dtype=np.float64)
    a = feature(D)
    S = mode_matrix(N, P.Wm.shape[1])
    C = P.Wl.shape[0]
    cache = Cache(u=u, a=a)
    h = P.Wl[None, :, 0, None, None] * u[:, None] + P.Wl[None, :, 1, None, None] * a[:, None, None, None] \
        + P.bl[None, :, None, None]
    cache.h.append(h)
    for l in range(P.Wm.shape[0]):
        T = np.einsum("bcyx,qx->bcyq", bf(h), bf(S))                  # contraction over x, bf16 operands
        hh = bf(np.einsum("py,bcyq->bcpq", S, T))
        gh = np.einsum("pqoc,bcpq->bopq", bf(P.Wm[l]), hh)
        Tf = np.einsum("bopq,qx->bopx", gh, S)
        z = np.einsum("py,bopx->boyx", bf(S), bf(Tf)) + np.einsum("oc,bcyx->boyx", bf(P.Wp[l]), bf(h)) \
            + P.bp[l][None, :, None, None]
        h = gelu(z)
        cache.hh.append(hh)
        cache.z.append(z)
        cache.h.append(h)
    assert h.shape[1] == C
    u_hat = u + np.einsum("c,bcyx->byx", P.Wq, h) + P.bq
    cache.rounding = rounding
    return u_hat, cache


def loss(u_hat: np.ndarray, target: np.ndarray) -> float:
    return float(np.mean((u_hat - target) ** 2))


def backward(P: Params, cache: Cache, u_hat: np.ndarray, target: np.ndarray, N: int) -> Params:
    """Gradient of the mean squared error with respect to every parameter."""
    S = mode_matrix(N, P.Wm.shape[1])
    g = zeros_like(P)
    du = 2.0 * (u_hat - target) / u_hat.size
    hL = cache.h[-1]
    g.Wq = np.einsum("byx,bcyx->c", du, hL)
    g.bq = np.array(du.sum())
    dh = P.Wq[None, :, None, None] * du[:, None]
    for l in reversed(range(P.Wm.shape[0])):
        h, z, hh = cache.h[l], cache.z[l], cache.hh[l]
        dz = dh * gelu_grad(z)
        g.bp[l] = dz.sum(axis=(0, 2, 3))
        g.Wp[l] = np.einsum("boyx,bcyx->oc", dz, h)
        dgh = np.einsum("py,boyx,qx->bopq", S, dz, S)
        g.Wm[l] = np.einsum("bopq,bcpq->pqoc", dgh, hh)
        Wm = bf16(P.Wm[l]) if getattr(cache, "rounding", True) else P.Wm[l]
        dhh = np.einsum("pqoc,bopq->bcpq", Wm, dgh)
        dh = np.einsum("oc,boyx->bcyx", P.Wp[l], dz) + np.einsum("py,bcpq,qx->bcyx", S, dhh, S)
    g.Wl[:, 0] = np.einsum("bcyx,byx->c", dh, cache.u)
    g.Wl[:, 1] = np.einsum("bcyx,b->c", dh, cache.a)
    g.bl = dh.sum(axis=(0, 2, 3))
    return g


@dataclass
class Adam:
    """Adam (Kingma and Ba 2015) with bias correction: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
    w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)."""
    lr: float = 1e-3
    b1: float = 0.9
    b2: float = 0.999
    eps: float = 1e-8
    t: int = 0
    m: Params = None
    v: Params = None

    def step(self, P: Params, g: Params) -> None:
        if self.m is None:
            self.m, self.v = zeros_like(P), zeros_like(P)
        self.t += 1
        c1, c2 = 1.0 - self.b1 ** self.t, 1.0 - self.b2 ** self.t
        for n in Params.NAMES:
            w, gr, m, v = getattr(P, n), getattr(g, n), getattr(self.m, n), getattr(self.v, n)
            m = self.b1 * m + (1.0 - self.b1) * gr
            v = self.b2 * v + (1.0 - self.b2) * gr * gr
            setattr(self.m, n, m)
            setattr(self.v, n, v)
            setattr(P, n, w - self.lr * (m / c1) / (np.sqrt(v / c2) + self.eps))


def parareal(u0: np.ndarray, windows: int, fine, coarse, iterations: int) -> list:
    """Parareal iterates for the initial value u0 over `windows` windows: U_0 = u0,
    U_{n+1}^{k+1} = G(U_n^{k+1}) + F(U_n^k) - G(U_n^k), starting from the coarse sweep U^0.
    fine / coarse map a state to the state one window later. Returns [U^0, U^1, ...], each a list
    of windows + 1 states."""
    U = [u0]
    for n in range(windows):
        U.append(coarse(U[n]))
    out = [U]
    for _ in range(iterations):
        Fk = [fine(U[n]) for n in range(windows)]
        Gk = [coarse(U[n]) for n in range(windows)]
        V = [u0]
        for n in range(windows):
            V.append(coarse(V[n]) + Fk[n] - Gk[n])
        U = V
        out.append(U)
    return out
