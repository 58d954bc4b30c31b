"""Batched executor (etd_batch_*): many independent 2D problems of uneven size in grouped launches.

A batch must reproduce one plan per problem to rounding (the batched kernel is its own
instantiation, so floating-point contraction may differ); problems are also checked against the
CPU oracle."""
import numpy as np
import pytest

from oracle import etd as oetd
from paper_2209_11922_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PROBLEMS = [((64, 96), 3e-3), ((96, 64), 1e-4), ((128, 384), 1e-2), ((384, 128), 5e-4), ((192, 256), 2e-3),
            ((256, 192), 7e-3), ((64, 64), 1e-2), ((96, 96), 1e-4), ((12, 8), 5e-2), ((6, 48), 1e-3)]


def _fields(problems, dtype, seed0=500):
    out = []
    for i, ((nx, ny), _) in enumerate(problems):
        U = inputs.uniform_field((ny - 1, nx - 1), -0.9, 0.9, seed=seed0 + i)
        out.append(torch.from_numpy(U.astype(np.float32 if dtype == "f32" else np.float64)).cuda())
    return out


@pytest.mark.parametrize("dtype,scheme", [("f32", 2), ("f64", 2), ("f32", 1)])
def test_batch_equals_one_plan_per_problem(dtype, scheme):
    from paper_2209_11922_gb300.etd import Batch, Plan
    tau, nsteps = 1e-2, 40     # one 32-step graph replay and 8 direct steps
    got = _fields(PROBLEMS, dtype)
    with Batch([p[0] for p in PROBLEMS], [p[1] for p in PROBLEMS], tau, scheme, dtype) as b:
        b.run(got, nsteps)
        info = b.info()
    assert info["launches_per_step"] >= 4 * scheme // 2
    ref = _fields(PROBLEMS, dtype)
    for (N, D), r in zip(PROBLEMS, ref):
        with Plan(N, D, tau, scheme=scheme, dtype=dtype) as pl:
            pl.run(r, nsteps)
    torch.cuda.synchronize()
    tol = 1e-5 if dtype == "f32" else 1e-13
    for i, (g, r) in enumerate(zip(got, ref)):
        g64, r64 = g.double(), r.double()
        rel = float((g64 - r64).norm() / r64.norm())
        assert rel <= tol, (i, PROBLEMS[i], rel)


def test_batch_schedules_give_identical_fields(monkeypatch):
    """The serial and the parallel-branch schedules run the same kernels on disjoint problems, so with the
    same tile sizes (the fixed choice, autotuning off) the fields agree bit for bit; the creation-time
    choice (autotuned tiles, both schedules timed) reports both trial times and keeps the faster, and its
    fields agree with the others to the FP32 bound (autotuned tiles may differ: results depend on the
    tile size at rounding level, see the design notes)."""
    from paper_2209_11922_gb300.etd import Batch
    tau, nsteps = 1e-2, 70     # two 32-step graph replays and 6 direct steps
    out = {}
    for sched in ("serial", "parallel", "auto"):
        with monkeypatch.context() as mp:
            if sched != "auto":
                mp.setenv("ETD_AUTOTUNE", "0")
            f = _fields(PROBLEMS, "f32", seed0=700)
            with Batch([p[0] for p in PROBLEMS], [p[1] for p in PROBLEMS], tau, 2, "f32", schedule=sched) as b:
                b.run(f, nsteps)
                out[sched] = (f, b.schedule(), b.info()["tile_pairs"])
    torch.cuda.synchronize()
    assert out["serial"][1]["schedule"] == "serial" and out["parallel"][1]["schedule"] == "parallel"
    assert out["serial"][2] == out["parallel"][2]
    for i, (a, b) in enumerate(zip(out["serial"][0], out["parallel"][0])):
        assert torch.equal(a, b), (i, PROBLEMS[i])
    auto = out["auto"][1]
    print(f"schedule trial: {auto}")
    assert auto["trial_us_per_step_serial"] > 0 and auto["trial_us_per_step_parallel"] > 0
    faster = "parallel" if auto["trial_us_per_step_parallel"] < auto["trial_us_per_step_serial"] else "serial"
    assert auto["schedule"] == faster
    for i, (a, b) in enumerate(zip(out["serial"][0], out["auto"][0])):
        rel = float((a.double() - b.double()).norm() / b.double().norm())
        assert rel <= 1e-5, (i, PROBLEMS[i], rel)


def test_batch_matches_oracle():
    from paper_2209_11922_gb300.etd import Batch
    probs = [((96, 64), 2e-3), ((64, 128), 1e-2), ((384, 96), 1e-4)]
    tau, nsteps = 1e-2, 10
    fields = _fields(probs, "f32", seed0=900)
    U0 = [f.cpu().numpy().astype(np.float64) for f in fields]
    with Batch([p[0] for p in probs], [p[1] for p in probs], tau, 2, "f32") as b:
        b.run(fields, nsteps)
    for (N, D), u0, f in zip(probs, U0, fields):
        ref = oetd.run(u0, N, (1 / N[0], 1 / N[1]), D, tau, nsteps, 2)
        got = f.cpu().numpy().astype(np.float64)
        l2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        linf = np.abs(got - ref).max() / np.abs(ref).max()
        assert l2 <= 1e-5 and linf <= 1e-5, (N, l2, linf)


def test_batch_run_twice_continues_and_zero_steps_is_noop():
    from paper_2209_11922_gb300.etd import Batch
    probs = PROBLEMS[:4]
    a = _fields(probs, "f64")
    b_ = _fields(probs, "f64")
    with Batch([p[0] for p in probs], [p[1] for p in probs], 1e-2, 2, "f64") as b:
        b.run(a, 20)
        b.run(b_, 7)
        b.run(b_, 0)
        b.run(b_, 13)
    for x, y in zip(a, b_):   # split runs agree to rounding (one extra transform round trip)
        assert torch.allclose(x, y, rtol=0, atol=1e-12 * float(x.abs().max()))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_periodic_batch_matches_oracle(dtype):
    """A periodic batch (Hartley kernels) with the Flory-Huggins reaction of Example 5.3, problems of
    uneven size, against the oracle's periodic path."""
    from paper_2209_11922_gb300.etd import Batch
    probs = [((96, 64), 1e-4), ((64, 128), 1e-3), ((384, 96), 1e-4), ((6, 48), 2e-3)]
    tau, nsteps = 20 / 2048, 8
    fh = dict(flin=1.6, fcub=0.0, flog=-0.8)
    U0 = [inputs.uniform_field((ny, nx), -0.9, 0.9, seed=950 + i) for i, ((nx, ny), _) in enumerate(probs)]
    if dtype == "f32":
        U0 = [u.astype(np.float32).astype(np.float64) for u in U0]
    fields = [torch.from_numpy(u.astype(np.float32 if dtype == "f32" else np.float64)).cuda() for u in U0]
    with Batch([p[0] for p in probs], [p[1] for p in probs], tau, 2, dtype, bc="periodic", **fh) as b:
        b.run(fields, nsteps)
    tol = 1e-5 if dtype == "f32" else 1e-12
    for (N, D), u0, f in zip(probs, U0, fields):
        ref = oetd.run(u0, N, (1 / N[0], 1 / N[1]), D, tau, nsteps, 2, bc="periodic", **fh)
        got = f.cpu().numpy().astype(np.float64)
        l2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        linf = np.abs(got - ref).max() / np.abs(ref).max()
        assert l2 <= tol and linf <= tol, (N, l2, linf)


def test_full_size_batch_sampled_problems_match_oracle():
    """The 512-problem workload (N_x, N_y from 64 to 384, D log-uniform in [1e-4, 1e-2], 200 ETDRK2 steps, FP32)
    in the launch configuration the bench times (tile sizes and schedule tuned at creation, graph replay), with
    one sampled problem per x length checked against the FP64 oracle over the whole run (T = 2).

    Bound 1e-4 (the batched workload's stated target is a final-time rel L2 <= 1e-3). Over T = 2 the FP32 floor
    exceeds the 1e-5 of shorter runs: Allen-Cahn amplifies rounding at rate f'(0) = 1 where diffusion is weak,
    and even the odd-extension transforms (rounding ~ log N) measure up to 1.8e-5 on these problems; the
    default FP32 route below N = 512 is the half-length recurrence (rounding ~ sqrt(N/2) eps), measured up to
    4.6e-5. One plan per problem on the same route gives the same errors (the batch adds nothing); both are
    reported next to the odd-extension plan's."""
    from paper_2209_11922_gb300.etd import Batch, Plan
    bw = inputs.BATCH_2D_512
    probs = bw.problems()
    shapes = [(ny - 1, nx - 1) for (nx, ny), _ in probs]
    U0 = [bw.u0(i, s).astype(np.float32) for i, s in enumerate(shapes)]
    fields = [torch.from_numpy(u).cuda() for u in U0]
    with Batch([p[0] for p in probs], [p[1] for p in probs], bw.tau, 2, "f32") as b:
        b.run(fields, bw.nsteps)
        torch.cuda.synchronize()
    sample, seen = [], set()
    for i, ((nx, ny), _) in enumerate(probs):
        if nx not in seen:
            seen.add(nx)
            sample.append(i)
    assert len(sample) == 6
    rows = []
    for i in sample:
        (N, D) = probs[i]
        ref = oetd.run(U0[i].astype(np.float64), N, (1 / N[0], 1 / N[1]), D, bw.tau, bw.nsteps, 2)
        errs = {}
        for name, route in (("batch", None), ("plan", "auto"), ("plan_odd", "fft")):
            if route is None:
                got = fields[i].cpu().numpy().astype(np.float64)
            else:
                with Plan(N, D, bw.tau, 2, "f32", route=route) as pl:
                    u = torch.from_numpy(U0[i]).cuda()
                    pl.run(u, bw.nsteps)
                    got = u.cpu().numpy().astype(np.float64)
            errs[name] = (np.linalg.norm(got - ref) / np.linalg.norm(ref), np.abs(got - ref).max() / np.abs(ref).max())
        rows.append((i, N, D, errs))
        print(f"problem {i} N={N} D={D:.2e}: " + ", ".join(f"{k} rel L2 {v[0]:.2e} Linf {v[1]:.2e}" for k, v in errs.items()))
    for i, N, D, errs in rows:
        assert max(errs["batch"]) <= 1e-4, (i, N, D, errs)
