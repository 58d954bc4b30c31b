"""Throughput of the EIFE2 (ETDRK2) Q1 finite-element solve on GB300, one JSON line on stdout.

A bench "step" is one full run of the workload: the 2D Allen-Cahn field on a 1024 x 1024 mesh
(1023^2 interior unknowns, D = 1e-4, tau = 5e-3, FP32 transforms with FP64-derived tables) advanced
by 2000 ETDRK2 time steps from its seeded synthetic u0, which is resident in HBM when timing starts.
value = unknown-updates per second (unknowns x time steps / s) over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference] [--workload NAME]

--impl reference times the CPU oracle (the plain FP64 NumPy implementation that the tests use as
ground truth) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2209_11922_gb300 import inputs  # noqa: E402

METRIC = "ETDRK2 unknown-updates/s"
UNIT = "unknown-updates/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Sources of the FFT-route pass kernels and of their launch configuration and tables: a change to any
# of them voids the DRAM-traffic record of profiles/traffic.json.
PASS_KERNEL_SOURCES = ("dst_engine.cuh", "pass_kernel.cuh", "etd_coeffs.cuh", "etd_api.cu")


def _kernel_source_hash() -> str:
    import hashlib
    d = os.path.join(ROOT, "paper_2209_11922_gb300", "csrc")
    h = hashlib.sha256()
    for f in PASS_KERNEL_SOURCES:
        h.update(f.encode())
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def _traffic(key: str):
    """DRAM bytes per launch recorded from an ncu capture, or None if the kernels changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            t = json.load(fh)
        if t.get("source_hash") != _kernel_source_hash():
            return None
        return t["entries"].get(key)
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _job_throughput(ms_local: float, updates_per_rank: float, world: int, device: str = "cuda"):
    """Whole-job throughput of `world` replicas: the slowest rank's time (max over ranks, one
    all-reduce; the caller brackets the timed region with barriers) and the updates of all ranks
    divided by it. Returns (ms_max, updates_per_s)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, updates_per_rank * world / (ms_max * 1e-3)


def _job_e2e(per_rank_value: float, world: int, device: str = "cuda") -> float:
    """End-to-end whole-job throughput: the slowest rank's rate times the number of ranks."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(per_rank_value)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MIN)
    return float(t.item()) * world


def _dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args, w):
    """The CPU oracle on a bounded sample of the workload (rank 0 only)."""
    world, rank, _ = _dist_setup(args)
    if rank != 0:
        return 0
    sample = args.ref_sample_steps
    u0 = w.u0()
    st, f = _oracle_stepper(w)
    for _ in range(args.warmup):
        st.run(u0, sample, f)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st.run(u0, sample, f)
    dt = time.perf_counter() - t0
    value = w.unknowns * sample * args.steps / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count() or 1)))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "sample": f"{sample} time steps of the {w.N} field per bench step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{sample} ETDRK2 time steps of {w.name} per step, {args.steps} steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _oracle_stepper(w):
    """The oracle's stepper and reaction for workload w (boundary condition and reaction included)."""
    from oracle import etd as oetd
    st = oetd.make_stepper(w.N, w.h, w.D, w.tau, w.scheme, 0.5, w.bc)
    f = oetd.reaction(w.flin, w.fcub, w.flog) if w.flog else oetd.allen_cahn(w.flin, w.fcub)
    return st, f


def cpu_baseline(w, seconds: float = 15.0) -> dict:
    """Time the oracle on the host cores for a bounded sample of the same workload."""
    u0 = w.u0()
    st, f = _oracle_stepper(w)
    t0 = time.perf_counter()
    st.run(u0, 1, f)
    one = time.perf_counter() - t0
    n = max(1, min(200, int(seconds / max(one, 1e-3))))
    t0 = time.perf_counter()
    st.run(u0, n, f)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count() or 1)))
    return {"value": w.unknowns * n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} ETDRK2 time steps of {w.name} (FP64 NumPy oracle, dense per-axis products)"}


def run_gb300(args, w):
    import torch
    import torch.distributed as dist

    from paper_2209_11922_gb300.etd import Plan

    world, rank, local = _dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dtype = args.dtype
    tdt = torch.float32 if dtype == "f32" else torch.float64
    nsteps = args.time_steps or w.nsteps
    plan = Plan(w.N, w.D, w.tau, scheme=w.scheme, dtype=dtype, route=args.route, bc=w.bc, flin=w.flin,
                fcub=w.fcub, flog=w.flog)
    info = plan.info()
    u0 = torch.from_numpy(w.u0().astype(np.float32 if dtype == "f32" else np.float64)).cuda()
    u = torch.empty_like(u0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def one_run():
        u.copy_(u0)
        flush.fill_(1.0)                         # evict L2 between bench steps
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.run(u, nsteps, stream)
        e1.record(stream)
        return e0, e1

    for _ in range(args.warmup):
        one_run()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    evs = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            evs.append(one_run())
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    ms_max, value = _job_throughput(ms, float(w.unknowns) * nsteps * args.steps, world)
    nonfinite = plan.monitor(u)["nonfinite"]

    # kernel-level timing of the same workload (separate run, events around every launch)
    u.copy_(u0)
    prof = plan.run_profiled(u, min(nsteps, 200), stream)
    kinds = {k: v for k, v in prof.items() if v[1] > 0}
    step_kinds = {k: v for k, v in kinds.items() if k not in ("entry_exit", "pack", "monitor")}
    dom = max(step_kinds, key=lambda k: step_kinds[k][0])
    dom_ms, dom_n = step_kinds[dom]
    # the FFT routes keep the state also transformed along the last axis: their closing stage pass writes
    # it as a second output (the split-radix route, whose last axis has no such pass, and the GEMM
    # routes do not)
    spec = args.route in ("auto", "fft", "fft_half")
    rw = {"x_react": 2, "transform": 2, "stage1_etdrk2": 4, "stage2_etdrk2": 4 if spec else 3,
          "stage_etdrk1": 4 if spec else 3}[dom]
    esz = 4 if dtype == "f32" else 8
    alg_bytes = rw * w.unknowns * esz
    achieved = alg_bytes / (dom_ms * 1e-3 / dom_n) / 1e9
    peak, peak_src = _peaks()
    traffic = _traffic(f"{w.name}:{dtype}:{args.route}:{dom}")

    # end to end through the C ABI with host buffers (copies inside the timed region)
    hbuf = torch.empty(u0.shape, dtype=tdt, pin_memory=True).numpy()
    u0h = u0.cpu().numpy()
    for _ in range(max(1, args.warmup)):
        hbuf[...] = u0h
        plan.run_host(hbuf, nsteps)
    e2e_t = 0.0
    for _ in range(args.steps):
        hbuf[...] = u0h
        t0 = time.perf_counter()
        plan.run_host(hbuf, nsteps)
        e2e_t += time.perf_counter() - t0
    e2e_val = _job_e2e(float(w.unknowns) * nsteps * args.steps / e2e_t, world)

    if rank == 0:
        clocks = clk.summary()
        # entry + exit launches per run (2D: entry, last-axis transform of the state, exit; 3D: two more)
        entry_exit = (2 if len(w.N) == 2 else 4) + (1 if spec else 0)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": w.name, "route": args.route, "mesh": list(w.N), "unknowns": w.unknowns, "time_steps_per_step": nsteps,
                       "D": w.D, "tau": w.tau, "scheme": "ETDRK2" if w.scheme == 2 else "ETDRK1",
                       "bc": w.bc, "reaction": {"flin": w.flin, "fcub": w.fcub, "flog": w.flog},
                       "parallelism": f"replicas x{world}",
                       "l2": "256 MiB buffer written between bench steps; within one run the fields stay L2-resident",
                       "kernels_per_time_step": info["kernels_per_step"],
                       "ms_per_time_step": ms_max / args.steps / nsteps},
            "gpu_launches": args.steps * (info["kernels_per_step"] * nsteps + entry_exit),
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_src, "traffic": traffic,
                         "alg_bytes_per_launch": alg_bytes, "launch_ms": dom_ms / dom_n,
                         "timing": "CUDA events around every launch of a separate profiled run"},
            "pass_ms": {k: round(v[0] / max(v[1], 1), 5) for k, v in kinds.items()},
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": w.unknowns * esz,
                    "d2h_bytes_per_step": w.unknowns * esz},
            "clocks": clocks,
            "nonfinite": nonfinite,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
        if world == 1 and not args.no_extras and w is inputs.AC2D_1024:
            # the other configurations of the workload set, measured after the headline (outside its
            # timed region): 256^3 on every route, the split-radix route, the batch and the surrogate
            line["route_fft_split_2d_1024"] = measure_split_route(args)
            line["config2_arms"] = measure_config2_arms(args)
            line["config3_3d_256cubed"] = measure_3d(args)
            line["config4_batched"] = measure_batched(args, inputs.BATCH_2D_512, 3, 3)
            sno = measure_sno(args, inputs.SNO_256)
            line["config5_surrogate"] = {k: sno[k] for k in (
                "metric", "value", "unit", "config", "plain_ms", "parareal_sno_ms", "parareal_sno", "final_rel_l2_sno",
                "parareal_etdrk2_coarse_ms", "parareal_etdrk2_coarse", "final_rel_l2_etdrk2",
                "gain_vs_nonlearned_coarse", "coarse_sno_ms", "roofline") if k in sno}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    plan.close()
    return 0


def measure_batched(args, bw, steps: int, warmup: int, nsteps: int = 0) -> dict:
    """Many independent 2D problems advanced by one batch (grouped launches), against the same
    problems advanced one plan each (the plain GPU solver). Returns the measured figures, with the
    steady-state schedule the batch chose at creation and both schedules' trial times."""
    import torch

    from paper_2209_11922_gb300.etd import Batch, Plan

    probs = bw.problems()
    dtype = args.dtype
    npdt = np.float32 if dtype == "f32" else np.float64
    tdt = torch.float32 if dtype == "f32" else torch.float64
    shapes = [(ny - 1, nx - 1) for (nx, ny), _ in probs]
    sizes = [a * b for a, b in shapes]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    flat0 = torch.empty(int(offs[-1]), dtype=tdt, device="cuda")
    for i, shp in enumerate(shapes):
        flat0[int(offs[i]):int(offs[i + 1])] = torch.from_numpy(bw.u0(i, shp).astype(npdt).ravel()).cuda()
    flat = torch.empty_like(flat0)
    fields = [flat[int(offs[i]):int(offs[i + 1])].view(shp) for i, shp in enumerate(shapes)]
    unknowns = int(offs[-1])
    nsteps = nsteps or bw.nsteps
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    batch = Batch([p[0] for p in probs], [p[1] for p in probs], bw.tau, 2, dtype, route=args.route)
    create_s = time.perf_counter() - t0
    info = batch.info()
    sched = batch.schedule()

    def timed(fn, k):
        tot = 0.0
        for _ in range(k):
            flat.copy_(flat0)
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        return tot

    timed(lambda: batch.run(fields, nsteps, stream), warmup)
    ms = timed(lambda: batch.run(fields, nsteps, stream), steps)
    value = unknowns * nsteps * steps / (ms * 1e-3)
    # plain GPU solver: one plan per problem, run one after the other on the same stream
    plans = [Plan(N, D, bw.tau, 2, dtype, route=args.route) for N, D in probs]

    def run_plans():
        for pl, f in zip(plans, fields):
            pl.run(f, nsteps, stream)

    timed(run_plans, 1)
    psteps = max(1, steps // 2)
    ms_plans = timed(run_plans, psteps)
    value_plans = unknowns * nsteps * psteps / (ms_plans * 1e-3)
    for pl in plans:
        pl.close()
    batch.close()
    # Transform route per length: one N x N plan per distinct length of the batch on each route (the
    # tensor-core routes need N % 32 == 0), microseconds per time step and the route's rel L2 difference
    # from the FFT route after the same steps: what an FFT-versus-GEMM choice per length would pick from.
    per_len = {}
    if dtype == "f32":
        lengths = sorted({n for (nx, ny), _ in probs for n in (nx, ny)})
        for n in lengths:
            row, ref_u = {}, None
            u0 = torch.from_numpy(bw.u0(0, (n - 1, n - 1)).astype(np.float32)).cuda()
            for route in ("auto", "gemm_tf32", "gemm_bf16x3"):
                if route != "auto" and n % 32:
                    continue
                with Plan((n, n), 3e-3, bw.tau, 2, "f32", route=route) as pl:
                    u = u0.clone()
                    pl.run(u, 64, stream)
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    pl.run(u, 256, stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    row[route] = {"us_per_step": e0.elapsed_time(e1) * 1e3 / 256}
                    v = u0.clone()
                    pl.run(v, 20, stream)
                    if route == "auto":
                        ref_u = v.double()
                    else:
                        row[route]["rel_l2_vs_fft_20_steps"] = float((v.double() - ref_u).norm() / ref_u.norm())
            per_len[str(n)] = row
    esz = 4 if dtype == "f32" else 8
    achieved = 12 * unknowns * esz / (ms / steps / nsteps * 1e-3) / 1e9   # field passes per time step
    peak, peak_src = _peaks()
    return {"workload": bw.name, "problems": len(probs), "unknowns": unknowns, "time_steps_per_run": nsteps,
            "value": value, "unit": UNIT, "ms_per_run": ms / steps, "plans_value": value_plans,
            "speedup_vs_plans": value / value_plans, "launches_per_time_step": info["launches_per_step"],
            "tuned_tile_pairs": info["tile_pairs"], "schedule": sched, "create_s": round(create_s, 3),
            "route_per_length": per_len, "runs_timed": steps,
            # per run: entry (one group per x length), the state's y transform (one per y length), exit (per
            # x length), six lengths each
            "gpu_launches": steps * (info["launches_per_step"] * nsteps + 18),
            "roofline": {"bound": "hbm", "kernel": "one time step (all grouped launches)", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src,
                         "traffic": None}}


def run_batched(args, bw):
    """The batched workload as its own bench line."""
    import torch

    world, rank, local = _dist_setup(args)
    torch.cuda.set_device(local)
    with ClockSampler(local) as clk:
        m = measure_batched(args, bw, args.steps, args.warmup, args.time_steps)
    line = {
        "metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m["ms_per_run"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": bw.name, "problems": m["problems"], "unknowns": m["unknowns"],
                   "time_steps_per_step": m["time_steps_per_run"], "tau": bw.tau, "scheme": "ETDRK2",
                   "launches_per_time_step": m["launches_per_time_step"], "tuned_tile_pairs": m["tuned_tile_pairs"],
                   "schedule": m["schedule"], "create_s": m["create_s"],
                   "l2": "256 MiB buffer written between bench steps"},
        "gpu_launches": m["gpu_launches"], "plans_value": m["plans_value"],
        "speedup_vs_plans": m["speedup_vs_plans"], "route_per_length": m["route_per_length"],
        "roofline": m["roofline"], "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def measure_sno(args, sw) -> dict:
    """Parareal with the trained SNO as coarse propagator against the plain batched ETDRK2 solver on
    B problems at N x N (windows x window steps). Training (data from the plain solver, Adam) runs
    before the timed region. Also times Parareal with a non-learned coarse propagator (one ETDRK2
    step of window * tau) to show what the learning gains. Returns the bench line as a dict."""
    import torch

    from paper_2209_11922_gb300.etd import Batch
    from paper_2209_11922_gb300.sno import Parareal, Sno
    from paper_2209_11922_gb300.sno_train import make_pairs, rel_error, train

    world, rank, local = _dist_setup(args)
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    B, W, n = sw.batch, sw.windows, sw.N - 1
    ntraj = args.sno_trajectories or sw.trajectories
    t0 = time.perf_counter()
    u_in, u_out, Dtr = make_pairs(sw, range(ntraj))
    t_data = time.perf_counter() - t0
    nval = max(B, u_in.shape[0] // 20)
    sno = Sno(sw.N, sw.C, sw.M, sw.L, B)
    sno.set_params(sw.init_weights())
    t0 = time.perf_counter()
    hist = train(sno, u_in[nval:], u_out[nval:], Dtr[nval:], args.sno_epochs, B, lr=args.sno_lr, seed=sw.seed)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    val = rel_error(sno, u_in[:nval], u_out[:nval], Dtr[:nval], B)
    del u_in, u_out
    torch.cuda.empty_cache()
    # test problems: seeds beyond the training trajectories
    tid = [10 ** 6 + b for b in range(B)]
    D = [sw.D(i) for i in tid]
    u0 = torch.from_numpy(np.stack([sw.u0(i) for i in tid]).astype(np.float32)).cuda()
    plain = Batch([(sw.N, sw.N)] * B, D, sw.tau, 2, "f32")
    work = torch.empty_like(u0)
    steps = W * sw.window

    def run_plain():
        work.copy_(u0)
        plain.run([work[b] for b in range(B)], steps, stream)

    pr_sno = Parareal(sno, sw.N, D, sw.tau, sw.window, W)
    pr_big = Parareal(None, sw.N, D, sw.tau, sw.window, W)
    out = torch.empty_like(u0)
    stats = {}

    def run_pr(pr, key):
        _, st = pr.run(u0, W, args.sno_tol, 1e-2, out=out, stream=stream)
        stats[key] = st

    def timed(fn, k):
        tot = 0.0
        for _ in range(k):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / k

    timed(run_plain, args.warmup)
    ref = work.clone()
    with ClockSampler(local) as clk:
        ms_plain = timed(run_plain, args.steps)
        timed(lambda: run_pr(pr_sno, "sno"), args.warmup)
        ms_sno = timed(lambda: run_pr(pr_sno, "sno"), args.steps)
    err = lambda a: float(max((torch.linalg.vector_norm(a[b] - ref[b]) / torch.linalg.vector_norm(ref[b])).item()
                              for b in range(B)))
    err_sno = err(out)
    timed(lambda: run_pr(pr_big, "big"), 1)
    ms_big = timed(lambda: run_pr(pr_big, "big"), max(1, args.steps // 2))
    err_big = err(out)
    # the coarse propagator alone (one SNO application to B fields)
    g = torch.empty_like(u0)
    ms_coarse = timed(lambda: sno.forward(u0, D, out=g, stream=stream), args.steps)
    fl = 2.0 * B * sw.C * sw.L * (2 * (n * n * sw.M + n * sw.M * sw.M) + sw.C * n * n)   # GEMM flops
    # Algorithmic bytes of one inference forward (FP32 activations): lift (u in, h_0 out); per layer the
    # mesh contraction of the truncated transform (h in, T out), its second contraction (T in, modes
    # out), the mode mix (modes in and out), the first inverse contraction (modes in, T out), the second
    # (T in, z out) and the pointwise mix with GELU (h and z in, h' out); projection (h_L, u in, u_hat
    # out).
    npix, C, M, L = n * n, sw.C, sw.M, sw.L
    fwd_bytes = 4.0 * B * (npix + C * npix + L * (5 * C * npix + 4 * C * M * n + 4 * C * M * M) + C * npix + 2 * npix)
    hbm_peak, hbm_src = _peaks()
    achieved = fwd_bytes / (ms_coarse * 1e-3) / 1e9
    line = {
        "metric": "surrogate vs plain speedup at L2 err", "value": ms_plain / ms_sno, "unit": "x", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_sno, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (bf16 operands in the operator's contractions)", "data": "synthetic",
        "config": {"workload": sw.name, "problems": B, "mesh": [sw.N, sw.N], "windows": W,
                   "window_steps": sw.window, "tau": sw.tau, "channels": sw.C, "modes": sw.M, "layers": sw.L,
                   "train_trajectories": ntraj, "train_pairs": int(ntraj * W), "epochs": args.sno_epochs,
                   "train_s": round(t_train, 1), "data_s": round(t_data, 1),
                   "train_loss": [float("%.4g" % v) for v in hist], "val_rel_l2_one_window": val,
                   "tol": args.sno_tol, "fallback_tol": 1e-2},
        "plain_ms": ms_plain, "parareal_sno_ms": ms_sno, "parareal_sno": stats["sno"], "final_rel_l2_sno": err_sno,
        "parareal_etdrk2_coarse_ms": ms_big, "parareal_etdrk2_coarse": stats["big"], "final_rel_l2_etdrk2": err_big,
        "gain_vs_nonlearned_coarse": ms_big / ms_sno, "coarse_sno_ms": ms_coarse,
        "gpu_launches": None,
        "roofline": {"bound": "hbm", "kernel": "SNO forward, one application to B fields (bf16 tensor-core "
                     "contractions over the mesh, FP32 mode mix)", "achieved": achieved, "peak": hbm_peak,
                     "unit": "GB/s", "frac": achieved / hbm_peak, "peak_source": hbm_src, "traffic": None,
                     "alg_bytes": fwd_bytes, "contraction_tflops": fl / (ms_coarse * 1e-3) / 1e12},
        "clocks": clk.summary(),
    }
    for o in (pr_sno, pr_big, sno, plain):
        o.close()
    return line


def run_sno_parareal(args, sw):
    print(json.dumps(measure_sno(args, sw)), flush=True)
    return 0


def measure_3d(args) -> dict:
    """The 256^3 Allen-Cahn workload (255^3 unknowns, D = 1e-3, tau = 1e-2, ETDRK2, FP32) on each
    transform route: time per ETDRK2 step (events around a run of time steps after warm-up runs; the
    330 MB of fields exceed L2), unknown-updates/s, the step-level fraction of HBM bandwidth on the
    pass schedule's field passes (FFT routes 20 per step, GEMM routes 27, 4 bytes each), and the route's
    error against the oracle on the same configuration at 64^3 (63^3 unknowns, 5 steps)."""
    import torch

    from oracle import etd as oetd
    from paper_2209_11922_gb300.etd import Plan

    w, ws = inputs.AC3D_256, inputs.AC3D_64
    peak, peak_src = _peaks()
    nsteps = 20
    u0 = torch.from_numpy(w.u0().astype(np.float32)).cuda()
    U0s = ws.u0().astype(np.float32).astype(np.float64)
    ref = oetd.run(U0s, ws.N, ws.h, ws.D, ws.tau, 5, 2)
    ref_full = oetd.run(U0s, ws.N, ws.h, ws.D, ws.tau, ws.nsteps, 2)
    out = {"workload": w.name, "unknowns": w.unknowns, "time_steps_timed": nsteps,
           "error_case": f"{ws.name}, 5 steps, rel L2 / rel Linf against the FP64 oracle",
           "error_case_full": f"{ws.name}, the workload's {ws.nsteps} steps, rel L2 against the FP64 oracle",
           "routes": {}}
    stream = torch.cuda.current_stream()
    for route, passes in (("auto", 20), ("gemm_tf32", 27), ("gemm_bf16x3", 27)):
        with Plan(w.N, w.D, w.tau, 2, "f32", route=route) as pl:
            u = torch.empty_like(u0)
            for _ in range(2):
                u.copy_(u0)
                pl.run(u, nsteps, stream)
            torch.cuda.synchronize()
            ts = []
            for _ in range(3):
                u.copy_(u0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pl.run(u, nsteps, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) / nsteps)
            prof = pl.run_profiled(u, 4, stream)
        ms = min(ts)
        with Plan(ws.N, ws.D, ws.tau, 2, "f32", route=route) as pl:
            d = torch.from_numpy(U0s.astype(np.float32)).cuda()
            pl.run(d, 5)
            got = d.cpu().numpy().astype(np.float64)
            d.copy_(torch.from_numpy(U0s.astype(np.float32)))
            pl.run(d, ws.nsteps)
            got_full = d.cpu().numpy().astype(np.float64)
        achieved = passes * 4 * w.unknowns / (ms * 1e-3) / 1e9
        out["routes"][route] = {
            "ms_per_time_step": ms, "value": w.unknowns / (ms * 1e-3), "unit": UNIT,
            "field_passes_per_step": passes, "achieved_GBps": achieved, "peak": peak, "peak_source": peak_src,
            "frac": achieved / peak,
            "pass_ms": {k: round(v[0] / max(v[1], 1), 5) for k, v in prof.items() if v[1] > 0},
            "rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
            "rel_linf": float(np.abs(got - ref).max() / np.abs(ref).max()),
            "rel_l2_full": float(np.linalg.norm(got_full - ref_full) / np.linalg.norm(ref_full))}
    return out


_ORACLE_1024 = {}


def _oracle_1024(scheme: int) -> np.ndarray:
    """The FP64 oracle's first 100 steps of the 1023^2 workload from its FP32-rounded initial field."""
    from oracle import etd as oetd

    if scheme not in _ORACLE_1024:
        w = inputs.AC2D_1024
        U0 = w.u0().astype(np.float32).astype(np.float64)
        _ORACLE_1024[scheme] = oetd.run(U0, w.N, w.h, w.D, w.tau, 100, scheme)
    return _ORACLE_1024[scheme]


def measure_config2_arms(args) -> dict:
    """The 1023^2 workload's other arms (ETDRK1; FP64 transforms), beside the FP32 ETDRK2 headline: time per
    time step over a 200-step run after warm-up, and the error of the first 100 steps against the FP64
    oracle (rel L2 / rel Linf)."""
    import torch

    from paper_2209_11922_gb300.etd import Plan

    w = inputs.AC2D_1024
    stream = torch.cuda.current_stream()
    out = {"workload": w.name, "time_steps_timed": 200,
           "error_case": "first 100 steps, rel L2 / rel Linf against the FP64 oracle"}
    for dtype, scheme in (("f32", 1), ("f64", 2), ("f64", 1)):
        ref = _oracle_1024(scheme)
        U0 = w.u0().astype(np.float32).astype(np.float64 if dtype == "f64" else np.float32)
        with Plan(w.N, w.D, w.tau, scheme, dtype) as pl:
            u = torch.from_numpy(U0).cuda()
            pl.run(u, 100)
            got = u.cpu().numpy().astype(np.float64)
            u.copy_(torch.from_numpy(U0))
            pl.run(u, 40, stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pl.run(u, 200, stream)
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 200
        out[f"{dtype}_etdrk{scheme}"] = {
            "ms_per_time_step": ms, "value": w.unknowns / (ms * 1e-3), "unit": UNIT,
            "rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
            "rel_linf": float(np.abs(got - ref).max() / np.abs(ref).max())}
    return out


def measure_split_route(args) -> dict:
    """The headline workload on the split-radix FFT route against the default route: time per ETDRK2
    step over a 2000-step run and the error of 100 steps against the FP64 oracle, both routes."""
    import torch

    from paper_2209_11922_gb300.etd import Plan

    w = inputs.AC2D_1024
    U0 = w.u0().astype(np.float32)
    ref = _oracle_1024(2)
    stream = torch.cuda.current_stream()
    out = {"workload": w.name, "error_case": "100 ETDRK2 steps, rel L2 / rel Linf against the FP64 oracle"}
    for route in ("auto", "fft_split"):
        with Plan(w.N, w.D, w.tau, 2, "f32", route=route) as pl:
            u = torch.from_numpy(U0).cuda()
            pl.run(u, 100)
            got = u.cpu().numpy().astype(np.float64)
            for _ in range(2):
                u.copy_(torch.from_numpy(U0))
                pl.run(u, 200, stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pl.run(u, 2000, stream)
            e1.record(stream)
            torch.cuda.synchronize()
        out[route] = {"ms_per_time_step": e0.elapsed_time(e1) / 2000,
                      "rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                      "rel_linf": float(np.abs(got - ref).max() / np.abs(ref).max())}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=inputs.AC2D_1024.name,
                    choices=sorted(inputs.WORKLOADS) + sorted(inputs.BATCH_WORKLOADS) + sorted(inputs.SNO_WORKLOADS))
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--route", default="auto", choices=["auto", "fft", "fft_half", "fft_split", "gemm_tf32", "gemm_bf16x3"])
    ap.add_argument("--time-steps", type=int, default=0, help="override the workload's time-step count")
    ap.add_argument("--ref-sample-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other configurations (256^3 routes, split route, batch, surrogate)")
    ap.add_argument("--sno-trajectories", type=int, default=0, help="training trajectories (default: the workload's)")
    ap.add_argument("--sno-epochs", type=int, default=6)
    ap.add_argument("--sno-lr", type=float, default=1e-3)
    ap.add_argument("--sno-tol", type=float, default=1e-4, help="Parareal stopping correction")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.workload in inputs.BATCH_WORKLOADS:
        return run_batched(args, inputs.BATCH_WORKLOADS[args.workload])
    if args.workload in inputs.SNO_WORKLOADS:
        return run_sno_parareal(args, inputs.SNO_WORKLOADS[args.workload])
    w = inputs.WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)
    return run_gb300(args, w)


if __name__ == "__main__":
    sys.exit(main())
