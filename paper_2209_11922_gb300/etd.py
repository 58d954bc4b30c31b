"""Python binding of the C ABI: a plan object over device tensors (PyTorch for memory and streams).

Every step of the solve runs in the library's CUDA kernels; this module only checks shapes and
dtypes and passes pointers.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np

from . import _native as nat

_DT = {"f64": nat.ETD_F64, "f32": nat.ETD_F32}
_BC = {"dirichlet": nat.ETD_BC_DIRICHLET, "periodic": nat.ETD_BC_PERIODIC}
# batch steady-state schedule: timed at creation ("auto") or forced
_SCHEDULE = {"auto": 0, "serial": nat.ETD_DEBUG_BATCH_SERIAL, "parallel": nat.ETD_DEBUG_BATCH_PARALLEL}
_ROUTE = {"auto": nat.ETD_ROUTE_AUTO, "fft": nat.ETD_ROUTE_FFT, "fft_half": nat.ETD_ROUTE_FFT_HALF,
          "gemm_tf32": nat.ETD_ROUTE_GEMM_TF32, "gemm_bf16x3": nat.ETD_ROUTE_GEMM_BF16X3,
          "fft_split": nat.ETD_ROUTE_FFT_SPLIT}


def _torch():
    import torch
    return torch


def _stream_ptr(stream) -> Optional[int]:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Plan:
    """EIFE1/EIFE2 plan for u_t = D Lap u + flin u + fcub u^3 on a rectangle (2D or 3D).

    N: intervals per axis (N_x first); h: mesh sizes (default 1/N, the unit square/cube).
    Fields are torch tensors of shape (N_z-1, N_y-1, N_x-1) or (N_y-1, N_x-1), x fastest; with
    bc="periodic" every node is an unknown, (N_z, N_y, N_x) or (N_y, N_x).
    The reaction is f(u) = flin u + fcub u^3 + flog artanh(u) (Flory-Huggins, Example 5.3:
    flin = theta_c, fcub = 0, flog = -theta).
    """

    def __init__(self, N: Sequence[int], D: float, tau: float, scheme: int = 2, dtype: str = "f64",
                 h: Optional[Sequence[float]] = None, c2: float = 0.5, flin: float = 1.0, fcub: float = -1.0,
                 route: str = "auto", debug: int = 0, bc: str = "dirichlet", flog: float = 0.0):
        L = nat.lib()
        self.N = tuple(int(n) for n in N)
        self.ndim = len(self.N)
        self.h = tuple(float(x) for x in (h if h is not None else [1.0 / n for n in self.N]))
        if len(self.h) != self.ndim:
            raise ValueError("h must have one entry per axis")
        self.D, self.tau, self.scheme, self.dtype = float(D), float(tau), int(scheme), dtype
        opt = nat.EtdOptions()
        L.etd_options_default(ctypes.byref(opt))
        opt.dtype = _DT[dtype]
        opt.route = _ROUTE[route]
        opt.c2, opt.flin, opt.fcub, opt.flog = float(c2), float(flin), float(fcub), float(flog)
        opt.debug = int(debug)
        if bc not in _BC:
            raise ValueError("bc must be 'dirichlet' or 'periodic'")
        opt.bc = _BC[bc]
        self.bc = bc
        Na = (ctypes.c_int64 * 3)(*(list(self.N) + [1] * (3 - self.ndim)))
        ha = (ctypes.c_double * 3)(*(list(self.h) + [1.0] * (3 - self.ndim)))
        handle = ctypes.c_void_p()
        nat.check(L.etd_plan_create(ctypes.byref(handle), self.ndim, Na, ha, self.D, self.tau, self.scheme,
                                    ctypes.byref(opt)), "etd_plan_create")
        self._h = handle

    # ------------------------------------------------------------------ helpers
    @property
    def shape(self) -> tuple:
        cut = 0 if self.bc == "periodic" else 1
        return tuple(n - cut for n in reversed(self.N))

    @property
    def torch_dtype(self):
        torch = _torch()
        return torch.float32 if self.dtype == "f32" else torch.float64

    @property
    def np_dtype(self):
        return np.float32 if self.dtype == "f32" else np.float64

    def _check_field(self, u, name="u"):
        torch = _torch()
        if not isinstance(u, torch.Tensor) or not u.is_cuda:
            raise TypeError(f"{name} must be a CUDA torch.Tensor")
        if u.dtype != self.torch_dtype or tuple(u.shape) != self.shape or not u.is_contiguous():
            raise ValueError(f"{name} must be contiguous {self.torch_dtype} of shape {self.shape}")
        return ctypes.c_void_p(u.data_ptr())

    # ------------------------------------------------------------------ API
    def run(self, u, nsteps: int, stream=None, t0: float = 0.0):
        self._bnd_exc = None
        st = nat.lib().etd_run_from(self._h, self._check_field(u), int(nsteps), float(t0), _stream_ptr(stream))
        if st != nat.ETD_OK and getattr(self, "_bnd_exc", None) is not None:
            raise nat.EtdError(st, "etd_run_from (boundary callback)") from self._bnd_exc
        nat.check(st, "etd_run_from")
        return u

    def boundary_count(self) -> int:
        n = ctypes.c_int64()
        nat.check(nat.lib().etd_boundary_count(self._h, ctypes.byref(n)), "etd_boundary_count")
        return int(n.value)

    def boundary_nodes(self):
        """Full-grid node indices (ix, iy[, iz]) of the packed boundary layout of etd_set_boundary:
        faces x = 0, x = L_x, y = 0, y = L_y (, z = 0, z = L_z), each over all its nodes, x fastest."""
        Nx, Ny = self.N[0], self.N[1]
        if self.ndim == 2:
            iy = np.arange(Ny + 1)
            ix = np.arange(Nx + 1)
            xs = [np.zeros_like(iy), np.full_like(iy, Nx), ix, ix]
            ys = [iy, iy, np.zeros_like(ix), np.full_like(ix, Ny)]
            return np.concatenate(xs), np.concatenate(ys)
        Nz = self.N[2]
        zy = np.meshgrid(np.arange(Nz + 1), np.arange(Ny + 1), indexing="ij")
        zx = np.meshgrid(np.arange(Nz + 1), np.arange(Nx + 1), indexing="ij")
        yx = np.meshgrid(np.arange(Ny + 1), np.arange(Nx + 1), indexing="ij")
        xs, ys, zs = [], [], []
        for v in (0, Nx):
            xs.append(np.full(zy[0].size, v)); ys.append(zy[1].ravel()); zs.append(zy[0].ravel())
        for v in (0, Ny):
            xs.append(zx[1].ravel()); ys.append(np.full(zx[0].size, v)); zs.append(zx[0].ravel())
        for v in (0, Nz):
            xs.append(yx[1].ravel()); ys.append(yx[0].ravel()); zs.append(np.full(yx[0].size, v))
        return np.concatenate(xs), np.concatenate(ys), np.concatenate(zs)

    def set_boundary(self, fn):
        """Nonhomogeneous Dirichlet data: fn(t) -> (g, gdot), the boundary values and their time
        derivatives at time t in the packed layout of `boundary_nodes()`; None removes them."""
        L = nat.lib()
        if fn is None:
            nat.check(L.etd_set_boundary(self._h, nat.BOUNDARY_FN(), None), "etd_set_boundary")
            self._bnd_cb = None
            return
        count = self.boundary_count()

        def cb(t, gp, gdp, ctx):
            try:
                g, gd = fn(t)
                np.ctypeslib.as_array(gp, (count,))[:] = np.asarray(g, dtype=np.float64).reshape(count)
                np.ctypeslib.as_array(gdp, (count,))[:] = np.asarray(gd, dtype=np.float64).reshape(count)
                return 0
            except Exception as e:   # run() raises EtdError(ETD_ERR_INVALID_ARG) from it
                self._bnd_exc = e
                return 1

        c = nat.BOUNDARY_FN(cb)
        nat.check(L.etd_set_boundary(self._h, c, None), "etd_set_boundary")
        self._bnd_cb = c   # the library holds the pointer: keep the callback alive

    def set_source(self, amp: float, rate: float, *profiles):
        """Separable time-dependent source amp exp(-rate t) g_x[i] g_y[j] (g_z[k]) added to the reaction;
        one profile of N_a - 1 interior values per axis (periodic: N_a nodal values), x first; no
        profiles removes it."""
        L = nat.lib()
        if not profiles or all(g is None for g in profiles):
            nat.check(L.etd_set_source(self._h, 0.0, 0.0, None, None, None), "etd_set_source")
            return
        if len(profiles) != self.ndim:
            raise ValueError("one profile per axis")
        gs = [np.ascontiguousarray(g, dtype=np.float64) for g in profiles]
        for a, g in enumerate(gs):
            n = self.shape[self.ndim - 1 - a]
            if g.shape != (n,):
                raise ValueError(f"profile {a} must hold the {n} nodal values of axis {a}")
        P = ctypes.POINTER(ctypes.c_double)
        ptrs = [g.ctypes.data_as(P) for g in gs] + [None] * (3 - self.ndim)
        nat.check(L.etd_set_source(self._h, float(amp), float(rate), *ptrs), "etd_set_source")

    def step(self, u, stream=None):
        nat.check(nat.lib().etd_step(self._h, self._check_field(u), _stream_ptr(stream)), "etd_step")
        return u

    def run_host(self, u_host: np.ndarray, nsteps: int, stream=None) -> np.ndarray:
        """Host array in, host array out (copies in/out happen inside the library call)."""
        if not (isinstance(u_host, np.ndarray) and u_host.dtype == self.np_dtype and u_host.shape == self.shape
                and u_host.flags["C_CONTIGUOUS"]):
            raise ValueError(f"u_host must be a C-contiguous {self.np_dtype} array of shape {self.shape}")
        nat.check(nat.lib().etd_run_host(self._h, u_host.ctypes.data_as(ctypes.c_void_p), int(nsteps),
                                         _stream_ptr(stream)), "etd_run_host")
        return u_host

    def apply_dst(self, axis: int, inp, out=None, stream=None):
        torch = _torch()
        if out is None:
            out = torch.empty_like(inp)
        nat.check(nat.lib().etd_apply_dst(self._h, int(axis), self._check_field(inp, "in"),
                                          self._check_field(out, "out"), _stream_ptr(stream)), "etd_apply_dst")
        return out

    def monitor(self, u, stream=None) -> dict:
        m = nat.EtdMonitors()
        st = nat.lib().etd_monitor(self._h, self._check_field(u), ctypes.byref(m), _stream_ptr(stream))
        if st not in (nat.ETD_OK, nat.ETD_ERR_NONFINITE):
            nat.check(st, "etd_monitor")
        return {"mass": m.mass, "energy": m.energy, "maxabs": m.maxabs, "nonfinite": int(m.nonfinite),
                "status": st}

    def run_profiled(self, u, nsteps: int, stream=None) -> dict:
        ms = (ctypes.c_double * nat.ETD_NUM_PASS_KINDS)()
        cnt = (ctypes.c_int64 * nat.ETD_NUM_PASS_KINDS)()
        nat.check(nat.lib().etd_run_profiled(self._h, self._check_field(u), int(nsteps), _stream_ptr(stream), ms, cnt),
                  "etd_run_profiled")
        L = nat.lib()
        return {L.etd_pass_kind_name(k).decode(): (ms[k], int(cnt[k])) for k in range(nat.ETD_NUM_PASS_KINDS)}

    def info(self) -> dict:
        i = nat.EtdPlanInfo()
        nat.check(nat.lib().etd_get_plan_info(self._h, ctypes.byref(i)), "etd_get_plan_info")
        return {"ndim": i.ndim, "N": tuple(i.N[:i.ndim]), "unknowns": i.unknowns,
                "workspace_bytes": i.workspace_bytes, "kernels_per_step": i.kernels_per_step,
                "bytes_per_step": i.bytes_per_step, "dtype": i.dtype, "scheme": i.scheme}

    def close(self):
        if getattr(self, "_h", None):
            nat.lib().etd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Many independent 2D problems advanced together (etd_batch_*): per problem its own
    intervals N_i = (N_x, N_y), mesh sizes (default 1/N) and diffusion D_i; common tau, scheme and
    options. Fields are a list of CUDA tensors of shape (N_y - 1, N_x - 1) (periodic: (N_y, N_x))."""

    def __init__(self, N: Sequence[Sequence[int]], D: Sequence[float], tau: float, scheme: int = 2,
                 dtype: str = "f32", h: Optional[Sequence[Sequence[float]]] = None, c2: float = 0.5,
                 flin: float = 1.0, fcub: float = -1.0, route: str = "auto", bc: str = "dirichlet",
                 flog: float = 0.0, schedule: str = "auto"):
        L = nat.lib()
        if schedule not in _SCHEDULE:
            raise ValueError(f"schedule must be one of {sorted(_SCHEDULE)}")
        self.N = [tuple(int(v) for v in n) for n in N]
        self.count = len(self.N)
        self.h = [tuple(float(v) for v in x) for x in (h if h is not None else [(1.0 / a, 1.0 / b) for a, b in self.N])]
        self.D = [float(d) for d in D]
        self.dtype = dtype
        if len(self.D) != self.count or len(self.h) != self.count:
            raise ValueError("N, h and D need one entry per problem")
        opt = nat.EtdOptions()
        L.etd_options_default(ctypes.byref(opt))
        opt.dtype, opt.route = _DT[dtype], _ROUTE[route]
        opt.c2, opt.flin, opt.fcub, opt.flog = float(c2), float(flin), float(fcub), float(flog)
        if bc not in _BC:
            raise ValueError("bc must be 'dirichlet' or 'periodic'")
        opt.bc = _BC[bc]
        opt.debug = _SCHEDULE[schedule]
        self.bc = bc
        Na = (ctypes.c_int64 * (2 * self.count))(*[v for n in self.N for v in n])
        ha = (ctypes.c_double * (2 * self.count))(*[v for x in self.h for v in x])
        Da = (ctypes.c_double * self.count)(*self.D)
        handle = ctypes.c_void_p()
        nat.check(L.etd_batch_create(ctypes.byref(handle), self.count, Na, ha, Da, float(tau), int(scheme),
                                     ctypes.byref(opt)), "etd_batch_create")
        self._h = handle

    def shapes(self):
        cut = 0 if self.bc == "periodic" else 1
        return [(ny - cut, nx - cut) for nx, ny in self.N]

    def run(self, fields, nsteps: int, stream=None):
        torch = _torch()
        tdt = torch.float32 if self.dtype == "f32" else torch.float64
        if len(fields) != self.count:
            raise ValueError("one field per problem")
        for f, shp in zip(fields, self.shapes()):
            if not (isinstance(f, torch.Tensor) and f.is_cuda and f.dtype == tdt and tuple(f.shape) == shp
                    and f.is_contiguous()):
                raise ValueError(f"fields must be contiguous CUDA {tdt} tensors of shapes {self.shapes()[:3]}...")
        ptrs = (ctypes.c_void_p * self.count)(*[f.data_ptr() for f in fields])
        nat.check(nat.lib().etd_batch_run(self._h, ptrs, int(nsteps), _stream_ptr(stream)), "etd_batch_run")
        return fields

    def info(self) -> dict:
        unk = ctypes.c_int64()
        nl = ctypes.c_int()
        tiles = (ctypes.c_int * 64)()
        nat.check(nat.lib().etd_batch_info(self._h, ctypes.byref(unk), ctypes.byref(nl), tiles, 64), "etd_batch_info")
        return {"unknowns": unk.value, "launches_per_step": nl.value, "tile_pairs": list(tiles[:min(nl.value, 64)])}

    def schedule(self) -> dict:
        """The steady-state schedule chosen at creation and the trial's microseconds per step of each."""
        par = ctypes.c_int()
        us = (ctypes.c_double(), ctypes.c_double())
        nat.check(nat.lib().etd_batch_schedule(self._h, ctypes.byref(par), ctypes.byref(us[0]), ctypes.byref(us[1])),
                  "etd_batch_schedule")
        return {"schedule": "parallel" if par.value else "serial", "trial_us_per_step_serial": us[0].value,
                "trial_us_per_step_parallel": us[1].value}

    def close(self):
        if getattr(self, "_h", None):
            nat.lib().etd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
