"""Tensor-core (GEMM) transform routes against the CPU oracle, through the C ABI.

Tolerances come from the operand precision of each route.
  gemm_tf32    TF32 operands keep 10 stored mantissa bits, u = 2^-10 (truncation). A transform
               y = S x with S and x each carrying a relative error u has relative error about 2u;
               the bound allows 5 x 2u = 9.8e-3 (measured 1.6e-3 to 2.8e-3).
  gemm_bf16x3  x = hi + lo and S = hi + lo in bf16 pairs (8 significant bits each, rounded to
               nearest): |x - hi| <= 2^-8 |x| and |x - hi - lo| <= 2^-8 |x - hi| <= 2^-16 |x|, and
               the products keep hi*hi + hi*lo + lo*hi, dropping lo*lo (<= 2^-16 |x||s|). Each
               transform therefore carries a worst-case relative error of about 2u, u = 2^-16, i.e.
               3.05e-5, which is the bound (measured 9.0e-6 to 1.43e-5 over these runs: the
               per-element errors are random in sign and diffusion damps rather than amplifies
               them over these short runs, so the multi-step error stays below one transform's
               worst case). A dropped hi*lo product would add 2^-8 relative error and fail it.
These runs are short (<= 10 steps).
"""
import numpy as np
import pytest

from oracle import etd as oetd
from paper_2209_11922_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROUTES = ("gemm_tf32", "gemm_bf16x3")
TOL = {"gemm_tf32": 5 * 2 * 2.0 ** -10, "gemm_bf16x3": 2 * 2.0 ** -16}


def _plan(N, D, tau, scheme=2, route="gemm_tf32", **kw):
    from paper_2209_11922_gb300.etd import Plan
    return Plan(N, D, tau, scheme=scheme, dtype="f32", route=route, **kw)


def _rel(got, ref):
    got = np.asarray(got, dtype=np.float64)
    l2 = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
    linf = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)
    return l2, linf


def _check(got, ref, route, what=""):
    l2, linf = _rel(got, ref)
    tol = TOL[route]
    assert l2 <= tol and linf <= tol, f"{route} {what}: rel L2 {l2:.3e} rel Linf {linf:.3e} (tol {tol:.1e})"
    return l2, linf


def _u0(N, seed, lo=-0.9, hi=0.9):
    return inputs.uniform_field(inputs.interior_shape(N), lo, hi, seed).astype(np.float32).astype(np.float64)


CASES = [
    # N, D, tau, nsteps, scheme: several 128-row tiles and partial tiles, unequal axes, both schemes
    ((64, 64), 1e-2, 1e-2, 10, 2),
    ((64, 96), 1e-2, 1e-2, 5, 2),
    ((384, 128), 1e-3, 1e-2, 4, 2),
    ((64, 64), 1e-2, 1e-2, 10, 1),
    ((64, 64, 64), 1e-3, 1e-2, 3, 2),
    ((32, 64, 96), 1e-3, 1e-2, 3, 2),
    ((96, 32, 64), 1e-3, 1e-2, 2, 1),
    # extremes: the smallest axis (one 32-column K chunk, 32-wide tiles), the longest (K = 2048,
    # 64 chunks, the full per-column tables), a single partial row tile
    ((32, 32), 1e-2, 1e-2, 3, 2),
    ((2048, 32), 1e-4, 5e-3, 2, 2),
    ((32, 2048), 1e-4, 5e-3, 2, 2),
    ((32, 32, 32), 1e-2, 1e-2, 2, 2),
]


@pytest.mark.parametrize("route", ROUTES)
@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])) + f"_s{c[4]}")
def test_gemm_route_steps_match_oracle(route, case):
    N, D, tau, nsteps, scheme = case
    U0 = _u0(N, 31)
    ref = oetd.run(U0, N, [1.0 / n for n in N], D, tau, nsteps, scheme)
    with _plan(N, D, tau, scheme, route) as pl:
        assert pl.info()["kernels_per_step"] == 2 * len(N) * scheme
        d = torch.from_numpy(U0.astype(np.float32)).cuda()
        pl.run(d, nsteps)
        _check(d.cpu().numpy(), ref, route, str(N))


@pytest.mark.parametrize("route", ROUTES)
def test_gemm_route_sine_mode_decays(route):
    """f = 0: a product sine mode must decay by exp(-n tau D (mu_p + mu_q)) (Section 4)."""
    N, D, tau, n = (256, 256), 1e-3, 1e-2, 8
    x = np.arange(1, 256) / 256
    p, q = 3, 7
    U0 = np.outer(np.sin(q * np.pi * x), np.sin(p * np.pi * x))
    mu = lambda k: 6 * 256 ** 2 * (1 - np.cos(k * np.pi / 256)) / (2 + np.cos(k * np.pi / 256))
    ref = np.exp(-n * tau * D * (mu(p) + mu(q))) * U0
    with _plan(N, D, tau, 2, route, flin=0.0, fcub=0.0) as pl:
        d = torch.from_numpy(U0.astype(np.float32)).cuda()
        pl.run(d, n)
        _check(d.cpu().numpy(), ref, route, "sine mode")


@pytest.mark.parametrize("route", ROUTES)
def test_gemm_route_run_host_and_monitor(route):
    N, D, tau = (64, 96), 1e-2, 1e-2
    U0 = _u0(N, 32).astype(np.float32)
    with _plan(N, D, tau, 2, route) as pl:
        d = torch.from_numpy(U0.copy()).cuda()
        pl.run(d, 4)
        h = pl.run_host(U0.copy(), 4)
        assert np.array_equal(h, d.cpu().numpy())
        assert pl.monitor(d)["status"] == 0


@pytest.mark.parametrize("route", ROUTES)
def test_gemm_route_full_size_3d_256_first_step(route):
    w = inputs.AC3D_256
    U0 = w.u0().astype(np.float32).astype(np.float64)
    ref = oetd.run(U0, w.N, w.h, w.D, w.tau, 1, 2)
    with _plan(w.N, w.D, w.tau, 2, route) as pl:
        d = torch.from_numpy(U0.astype(np.float32)).cuda()
        pl.run(d, 1)
        _check(d.cpu().numpy(), ref, route, w.name)


@pytest.mark.parametrize("route", ROUTES)
def test_gemm_route_full_size_2d_1024_first_steps(route):
    w = inputs.AC2D_1024
    U0 = w.u0().astype(np.float32).astype(np.float64)
    ref = oetd.run(U0, w.N, w.h, w.D, w.tau, 3, 2)
    with _plan(w.N, w.D, w.tau, 2, route) as pl:
        d = torch.from_numpy(U0.astype(np.float32)).cuda()
        pl.run(d, 3)
        _check(d.cpu().numpy(), ref, route, w.name)


def test_gemm_pass_wait_limit_reports_timeout_and_leaves_the_context_usable():
    """Failure path of the tensor-core pass: with the debug option the first pass of a run never
    receives its accumulator-ready signal; its epilogue warps give up after their 2 s limit, the
    CTA frees its tensor memory and exits, and the next synchronising call reports
    ETD_ERR_TIMEOUT. Another plan then runs correctly on the same context."""
    from paper_2209_11922_gb300 import _native as nat
    N, D, tau = (64, 64), 1e-2, 1e-2
    U0 = _u0(N, 33).astype(np.float32)
    with _plan(N, D, tau, 2, "gemm_tf32", debug=nat.ETD_DEBUG_STALL_FIRST_GEMM_PASS) as pl:
        with pytest.raises(nat.EtdError) as ei:
            pl.run_host(U0.copy(), 1)
        assert ei.value.status == nat.ETD_ERR_TIMEOUT
    ref = oetd.run(U0.astype(np.float64), N, [1.0 / n for n in N], D, tau, 2, 2)
    with _plan(N, D, tau, 2, "gemm_tf32") as pl:
        _check(pl.run_host(U0.copy(), 2), ref, "gemm_tf32", "after a timed-out run")
