"""Periodic boundary conditions and the Flory-Huggins reaction on the GPU against the CPU oracle
(Section 4, closing remarks; Example 5.3 of Section 5.2), through the C ABI.

Tolerances as for the Dirichlet path: FP64 rel L2 and rel Linf <= 1e-12, FP32 <= 1e-5 over short
runs (the FP32 input is rounded first and the oracle runs on the rounded values in FP64). The
Flory-Huggins reaction has |f'| <= 8 on [-gamma, gamma]; over the few steps compared here that
amplifies the FP32 rounding of f by at most tau |f'| < 0.1 per step, inside the same bound.
"""
import numpy as np
import pytest

from oracle import etd as oetd
from oracle import monitors as omon
from oracle import transforms as otr
from paper_2209_11922_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
THETA, THETA_C = 0.8, 1.6
FH = dict(flin=THETA_C, fcub=0.0, flog=-THETA)


def _plan(N, D, tau, scheme=2, dtype="f64", **kw):
    from paper_2209_11922_gb300.etd import Plan
    return Plan(N, D, tau, scheme=scheme, dtype=dtype, bc="periodic", **kw)


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a.astype(np.float32 if dtype == "f32" else np.float64))).cuda()


def _u0(N, seed, dtype, lo=-0.9, hi=0.9):
    U = inputs.uniform_field(inputs.field_shape(N, "periodic"), lo, hi, seed)
    return U.astype(np.float32).astype(np.float64) if dtype == "f32" else U


def _check(got, ref, tol, what=""):
    got = np.asarray(got, dtype=np.float64)
    l2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    linf = np.abs(got - ref).max() / np.abs(ref).max()
    assert l2 <= tol and linf <= tol, f"{what}: rel L2 {l2:.3e} rel Linf {linf:.3e} (tol {tol:.0e})"


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("N", [(16, 12), (64, 96), (6, 8, 12), (32, 16, 24)])
def test_hartley_transform_matches_definition(N, dtype):
    U = _u0(N, 41, dtype, -1, 1)
    with _plan(N, 1e-2, 1e-2, dtype=dtype) as pl:
        for axis in range(len(N)):
            got = pl.apply_dst(axis, _dev(U, dtype)).cpu().numpy()
            _check(got, otr.dht_axis(U, axis), TOL[dtype], f"axis {axis}")


CASES = [
    # N, D, tau, nsteps, scheme, reaction: several tiles along every axis, unequal and 3*2^k axes
    ((64, 64), 1e-2, 1e-2, 8, 2, "ac"),
    ((96, 32), 1e-3, 2e-2, 6, 1, "ac"),
    ((128, 48), 1e-4, 20 / 2048, 8, 2, "fh"),
    ((256, 192), 1e-4, 20 / 2048, 4, 1, "fh"),
    ((16, 24, 32), 1e-3, 1e-2, 5, 2, "ac"),
    ((32, 32, 32), 1e-4, 20 / 2048, 6, 2, "fh"),
    ((48, 16, 8), 1e-4, 20 / 2048, 4, 1, "fh"),
    # extremes: the shortest and longest supported axes (4, 6 and 2048, 1536)
    ((4, 2048), 1e-4, 1e-2, 3, 2, "ac"),
    ((2048, 4), 1e-4, 20 / 2048, 3, 2, "fh"),
    ((1536, 6), 1e-4, 1e-2, 2, 1, "ac"),
    ((4, 6, 8), 1e-2, 1e-2, 3, 2, "fh"),
]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])) + f"_s{c[4]}_{c[5]}")
def test_periodic_steps_match_oracle(case, dtype):
    N, D, tau, nsteps, scheme, react = case
    h = tuple(1.0 / n for n in N)
    U0 = _u0(N, 43, dtype)
    kw = FH if react == "fh" else {}
    ref = oetd.run(U0, N, h, D, tau, nsteps, scheme, bc="periodic",
                   **({"flin": THETA_C, "fcub": 0.0, "flog": -THETA} if react == "fh" else {}))
    with _plan(N, D, tau, scheme, dtype, **kw) as pl:
        assert pl.shape == U0.shape
        d = _dev(U0, dtype)
        pl.run(d, nsteps)
        _check(d.cpu().numpy(), ref, TOL[dtype], str(N))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_fourier_mode_decays_exactly(dtype):
    """f = 0: a product Fourier mode decays by exp(-n tau D (mu_p + mu_q)), mu(theta = 2 pi k / N)."""
    N, D, tau, n = (128, 64), 2e-3, 0.05, 10
    x = np.arange(N[0]) / N[0]
    y = np.arange(N[1]) / N[1]
    U0 = np.outer(np.sin(2 * np.pi * 3 * y + 0.4), np.cos(2 * np.pi * 5 * x))
    mu = lambda k, m: 6 * m * m * (1 - np.cos(2 * np.pi * k / m)) / (2 + np.cos(2 * np.pi * k / m))
    ref = np.exp(-n * tau * D * (mu(5, N[0]) + mu(3, N[1]))) * U0
    with _plan(N, D, tau, 2, dtype, flin=0.0, fcub=0.0) as pl:
        d = _dev(U0, dtype)
        pl.run(d, n)
        _check(d.cpu().numpy(), ref, TOL[dtype], "Fourier mode")


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_periodic_monitors_match_oracle(dtype):
    N = (32, 24, 16)
    h = tuple(1.0 / n for n in N)
    D = 1e-4
    U = _u0(N, 44, dtype)
    ref = omon.monitors(U, N, h, D, "periodic", flory_huggins=(THETA, THETA_C))
    with _plan(N, D, 0.01, 2, dtype, **FH) as pl:
        m = pl.monitor(_dev(U, dtype))
    assert m["status"] == 0 and m["nonfinite"] == 0
    assert m["mass"] == pytest.approx(ref["mass"], rel=1e-12, abs=1e-14)
    assert m["energy"] == pytest.approx(ref["energy"], rel=1e-12)
    assert m["maxabs"] == ref["maxabs"]


def test_periodic_source_matches_oracle():
    """A separable source on a periodic plan (x profile transformed by the Hartley transform)."""
    N, D, tau, t0 = (32, 16), 0.02, 0.01, 0.2
    h = tuple(1.0 / n for n in N)
    x = np.arange(N[0]) * h[0]
    y = np.arange(N[1]) * h[1]
    gx, gy = np.cos(2 * np.pi * x) + 0.3 * np.sin(4 * np.pi * x), 1.0 + np.sin(2 * np.pi * y)
    G = np.outer(gy, gx)
    U0 = _u0(N, 45, "f64")

    def f(t, u):
        return u - u ** 3 + 1.5 * np.exp(-2.0 * t) * G

    ref = oetd.make_stepper(N, h, D, tau, 2, 0.5, "periodic").run(U0, 5, f, t0=t0)
    with _plan(N, D, tau, 2, "f64") as pl:
        pl.set_source(1.5, 2.0, gx, gy)
        d = _dev(U0, "f64")
        pl.run(d, 5, t0=t0)
        _check(d.cpu().numpy(), ref, 1e-12, "source")


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_example53_full_size_first_steps(dtype):
    """Example 5.3's configuration (128^3, periodic, Flory-Huggins, tau = 20/2048): the first steps
    element by element against the oracle at full size."""
    w = inputs.GC3D_128
    U0 = w.u0()
    if dtype == "f32":
        U0 = U0.astype(np.float32).astype(np.float64)
    ref = oetd.run(U0, w.N, w.h, w.D, w.tau, 2, 2, bc="periodic", flin=w.flin, fcub=w.fcub, flog=w.flog)
    with _plan(w.N, w.D, w.tau, 2, dtype, flin=w.flin, fcub=w.fcub, flog=w.flog) as pl:
        d = _dev(U0, dtype)
        pl.run(d, 2)
        _check(d.cpu().numpy(), ref, TOL[dtype], w.name)


def test_example53_whole_run_keeps_the_max_bound_and_decays_the_energy():
    """Example 5.3 in full on the GPU in FP64: 2048 EIFE2 steps to T = 20 on the 128^3 mesh. The
    supremum norm stays below gamma ~ 0.9575 and the energy decreases monotonically (the behaviour
    Section 5.2 reports for Figure 3), sampled every 32 steps."""
    w = inputs.GC3D_128
    g = omon.fh_max_bound(THETA, THETA_C)
    with _plan(w.N, w.D, w.tau, 2, "f64", flin=w.flin, fcub=w.fcub, flog=w.flog) as pl:
        d = _dev(w.u0(), "f64")
        m = pl.monitor(d)
        E, sup = [m["energy"]], [m["maxabs"]]
        for _ in range(w.nsteps // 32):
            pl.run(d, 32)
            m = pl.monitor(d)
            assert m["status"] == 0
            E.append(m["energy"])
            sup.append(m["maxabs"])
    # the bound holds in exact arithmetic; the converged phases sit at gamma itself, where FP64
    # rounding of the transforms leaves values a few ulp either side (1e-14 relative: ~90 ulp)
    assert max(sup) <= g * (1 + 1e-14)
    assert all(b <= a + 1e-12 * abs(a) for a, b in zip(E, E[1:]))
    assert sup[-1] > 0.95 * g          # the phases have separated
    assert E[-1] < 0.5 * E[0]


# ---------------------------------------------------------------- tensor-core routes (Hartley matrix)
GEMM_TOL = {"gemm_tf32": 5 * 2 * 2.0 ** -10, "gemm_bf16x3": 2 * 2.0 ** -16}   # as for the Dirichlet GEMM routes
GEMM_CASES = [
    ((64, 64), 1e-2, 1e-2, 5, 2, "ac"),
    ((64, 96), 1e-4, 20 / 2048, 4, 1, "fh"),
    ((32, 64, 96), 1e-4, 20 / 2048, 3, 2, "fh"),
    ((128, 128, 128), 1e-4, 20 / 2048, 2, 2, "fh"),
]


@pytest.mark.parametrize("route", ["gemm_tf32", "gemm_bf16x3"])
@pytest.mark.parametrize("case", GEMM_CASES, ids=lambda c: "x".join(map(str, c[0])) + f"_s{c[4]}_{c[5]}")
def test_periodic_gemm_routes_match_oracle(case, route):
    N, D, tau, nsteps, scheme, react = case
    h = tuple(1.0 / n for n in N)
    U0 = _u0(N, 47, "f32")
    kw = FH if react == "fh" else {}
    ref = oetd.run(U0, N, h, D, tau, nsteps, scheme, bc="periodic",
                   **({"flin": THETA_C, "fcub": 0.0, "flog": -THETA} if react == "fh" else {}))
    with _plan(N, D, tau, scheme, "f32", route=route, **kw) as pl:
        d = _dev(U0, "f32")
        pl.run(d, nsteps)
        _check(d.cpu().numpy(), ref, GEMM_TOL[route], f"{route} {N}")


@pytest.mark.parametrize("route", ["gemm_tf32", "gemm_bf16x3"])
def test_dirichlet_gemm_routes_take_the_artanh_term(route):
    """The GEMM routes apply f = flin u + fcub u^3 + flog artanh u on Dirichlet plans too."""
    from paper_2209_11922_gb300.etd import Plan
    N, D, tau, nsteps = (64, 96), 1e-3, 1e-2, 4
    h = tuple(1.0 / n for n in N)
    U0 = inputs.uniform_field(inputs.interior_shape(N), -0.9, 0.9, 48).astype(np.float32).astype(np.float64)
    ref = oetd.run(U0, N, h, D, tau, nsteps, 2, flin=THETA_C, fcub=0.0, flog=-THETA)
    with Plan(N, D, tau, scheme=2, dtype="f32", route=route, **FH) as pl:
        d = _dev(U0, "f32")
        pl.run(d, nsteps)
        _check(d.cpu().numpy(), ref, GEMM_TOL[route], f"{route} Dirichlet")


def test_periodic_zero_steps_is_a_no_op_and_split_runs_agree():
    N, D, tau = (64, 32, 16), 1e-4, 20 / 2048
    U0 = _u0(N, 49, "f64")
    with _plan(N, D, tau, 2, "f64", **FH) as pl:
        d = _dev(U0, "f64")
        pl.run(d, 0)
        assert np.array_equal(d.cpu().numpy(), U0)
        pl.run(d, 3)
        pl.run(d, 4)
        e = _dev(U0, "f64")
        pl.run(e, 7)
        _check(d.cpu().numpy(), e.cpu().numpy(), 1e-13, "3 + 4 vs 7 steps")
