"""The split-radix FP32 route (ETD_ROUTE_FFT_SPLIT: DST-I of N = 1024 as a DST-III of length 512, a
DST-III of length 256 and the odd extension of a DST-I of length 256, each on its own warp-level FFT)
against the definition of the transform and the CPU oracle, through the C ABI.

Bounds: FP32 1e-5 (rel L2 and rel Linf) for every run, including 100 steps at 1024^2; one transform
1e-6 (L2) / 3e-6 (Linf) against the definition (rounding grows like log N; measured 1.2e-7). The
linear-reaction cases check against the exact per-mode solution of EIFE2 for f = kappa u (eq. (2.14)
mode by mode): a strong reaction (kappa tau = -0.25) would amplify any coupling of the boundary row
or column into the transforms' zero-frequency terms, which once made modes N/4, N/2, 3N/4 grow by
~50x per step."""
import math

import numpy as np
import pytest
import scipy.fft as sfft

from oracle import etd as oetd
from oracle import transforms as otr
from paper_2209_11922_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def _plan(N, D, tau, scheme=2, **kw):
    from paper_2209_11922_gb300.etd import Plan
    return Plan(N, D, tau, scheme=scheme, dtype="f32", route="fft_split", **kw)


def _rel(got, ref):
    got = np.asarray(got, dtype=np.float64)
    return (np.linalg.norm(got - ref) / np.linalg.norm(ref), np.abs(got - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("N", [(1024, 8), (8, 1024), (1024, 1024), (4, 1024, 4), (8, 6, 1024)])
def test_split_dst_matches_definition(N):
    shape = tuple(n - 1 for n in reversed(N))
    U = inputs.uniform_field(shape, -1, 1, seed=sum(N)).astype(np.float32).astype(np.float64)
    with _plan(N, 0.1, 0.01) as pl:
        d = torch.from_numpy(U.astype(np.float32)).cuda()
        for axis in range(len(N)):
            if N[axis] != 1024:
                continue
            got = pl.apply_dst(axis, d).cpu().numpy()
            l2, linf = _rel(got, otr.dst_axis(U, axis))
            assert l2 <= 1e-6 and linf <= 3e-6, (N, axis, l2, linf)


@pytest.mark.parametrize("scheme,nsteps", [(2, 3), (1, 3), (2, 100)])
def test_split_full_size_2d_1024(scheme, nsteps):
    w = inputs.AC2D_1024
    U0 = w.u0().astype(np.float32).astype(np.float64)
    ref = oetd.run(U0, w.N, w.h, w.D, w.tau, nsteps, scheme)
    with _plan(w.N, w.D, w.tau, scheme) as pl:
        d = torch.from_numpy(U0.astype(np.float32)).cuda()
        pl.run(d, nsteps)
        l2, linf = _rel(d.cpu().numpy(), ref)
    assert l2 <= TOL and linf <= TOL, (scheme, nsteps, l2, linf)


def test_split_3d_with_a_1024_axis():
    N, D, tau, n = (8, 1024, 8), 1e-3, 1e-2, 4
    U0 = inputs.uniform_field((7, 1023, 7), -0.9, 0.9, seed=44).astype(np.float32).astype(np.float64)
    ref = oetd.run(U0, N, [1 / k for k in N], D, tau, n, 2)
    with _plan(N, D, tau) as pl:
        d = torch.from_numpy(U0.astype(np.float32)).cuda()
        pl.run(d, n)
        l2, linf = _rel(d.cpu().numpy(), ref)
    assert l2 <= TOL and linf <= TOL, (l2, linf)


def _exact_linear(Ut, D, tau, kappa, n, c2=0.5):
    """EIFE2 for f = kappa u, mode by mode: U~ -> R^n U~ (eq. (2.14) for one mode)."""
    k = np.arange(1, 1024)
    mu = 6 * 1024 ** 2 * (1 - np.cos(k * np.pi / 1024)) / (2 + np.cos(k * np.pi / 1024))
    Z = tau * D * (mu[None, :] + mu[:, None])
    phi1 = lambda w: np.expm1(w) / w
    phi2 = lambda w: (np.expm1(w) - w) / (w * w)
    kt = kappa * tau
    R = np.exp(-Z) + kt * (phi1(-Z) - phi2(-Z) / c2) + kt * (phi2(-Z) / c2) * (np.exp(-c2 * Z) + c2 * kt * phi1(-c2 * Z))
    return sfft.idstn(Ut * R ** n, type=1, norm="ortho")


@pytest.mark.parametrize("ymodes", [None, (511,), (256, 512, 768), (3,)], ids=["all", "511", "quarters", "3"])
def test_split_linear_reaction_matches_exact_modes(ymodes):
    """Random x content on a set of y modes (all modes: a white-noise field), f = -50 u, 4 EIFE2 steps."""
    D, tau, kappa, n = 1e-4, 5e-3, -50.0, 4
    rng = np.random.default_rng(3)
    Ut = sfft.dstn(rng.uniform(-1, 1, (1023, 1023)), type=1, norm="ortho")
    if ymodes is not None:
        keep = np.zeros(1023, bool)
        keep[[m - 1 for m in ymodes]] = True
        Ut[~keep, :] = 0
    u0 = sfft.idstn(Ut, type=1, norm="ortho").astype(np.float32)
    Ut = sfft.dstn(u0.astype(np.float64), type=1, norm="ortho")
    ref = _exact_linear(Ut, D, tau, kappa, n)
    with _plan((1024, 1024), D, tau, flin=kappa, fcub=0.0) as pl:
        d = torch.from_numpy(u0).cuda()
        pl.run(d, n)
        got = d.cpu().numpy().astype(np.float64)
    # high modes decay ~1000x over the run: errors are measured against max(||ref||, 0.1 ||u0||) so that
    # rounding at the scale of u0 is not read as an error of the decayed field
    scale2 = max(np.linalg.norm(ref), 0.1 * np.linalg.norm(u0))
    scalei = max(np.abs(ref).max(), 0.1 * np.abs(u0).max())
    l2, linf = np.linalg.norm(got - ref) / scale2, np.abs(got - ref).max() / scalei
    assert l2 <= TOL and linf <= TOL, (ymodes, l2, linf)


def test_split_graph_replay_matches_direct_launches():
    w = inputs.AC2D_1024
    U0 = w.u0().astype(np.float32)
    with _plan(w.N, w.D, w.tau) as pl:
        a = torch.from_numpy(U0).cuda()
        pl.run(a, 40)            # one graph replay of 32 steps and 8 direct steps
        b = torch.from_numpy(U0).cuda()
        for _ in range(40):
            pl.step(b)           # direct launches, one entry/exit per step
        l2, linf = _rel(b.cpu().numpy(), a.cpu().numpy().astype(np.float64))
    assert l2 <= TOL and linf <= TOL, (l2, linf)
