"""Python binding of the spectral neural operator and the Parareal driver (include/etd_sno.h).

Argument marshalling only: every forward pass, gradient, Adam update, fine solve and correction
runs in the library's CUDA kernels. Fields are CUDA float32 torch tensors of shape (B, N-1, N-1).
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np

from . import _native as nat
from .etd import _stream_ptr, _torch

PARAM_NAMES = ("Wl", "bl", "Wm", "Wp", "bp", "Wq", "bq")


def param_shapes(C: int, M: int, L: int) -> dict:
    return {"Wl": (C, 2), "bl": (C,), "Wm": (L, M, M, C, C), "Wp": (L, C, C), "bp": (L, C), "Wq": (C,), "bq": ()}


def flatten(params: dict) -> np.ndarray:
    return np.concatenate([np.asarray(params[n], dtype=np.float32).reshape(-1) for n in PARAM_NAMES])


def unflatten(flat: np.ndarray, C: int, M: int, L: int) -> dict:
    out, off = {}, 0
    for n, shp in param_shapes(C, M, L).items():
        k = int(np.prod(shp)) if shp else 1
        out[n] = np.asarray(flat[off:off + k], dtype=np.float64).reshape(shp)
        off += k
    return out


def _darr(D: Sequence[float]):
    D = [float(d) for d in D]
    return (ctypes.c_double * len(D))(*D), len(D)


class Sno:
    """Operator for N x N meshes with C channels, M x M modes, L layers, batches <= max_batch."""

    def __init__(self, N: int, C: int, M: int, L: int, max_batch: int):
        self.N, self.C, self.M, self.L, self.max_batch = int(N), int(C), int(M), int(L), int(max_batch)
        h = ctypes.c_void_p()
        nat.check(nat.lib().etd_sno_create(ctypes.byref(h), self.N, self.C, self.M, self.L, self.max_batch),
                  "etd_sno_create")
        self._h = h
        self.nparam = int(nat.lib().etd_sno_param_count(h))

    def set_params(self, params: dict):
        flat = np.ascontiguousarray(flatten(params))
        if flat.size != self.nparam:
            raise ValueError(f"expected {self.nparam} parameters, got {flat.size}")
        nat.check(nat.lib().etd_sno_set_params(self._h, flat.ctypes.data_as(ctypes.c_void_p)), "etd_sno_set_params")

    def get_params(self) -> dict:
        flat = np.empty(self.nparam, dtype=np.float32)
        nat.check(nat.lib().etd_sno_get_params(self._h, flat.ctypes.data_as(ctypes.c_void_p)), "etd_sno_get_params")
        return unflatten(flat, self.C, self.M, self.L)

    def _field(self, u, name="u"):
        torch = _torch()
        n = self.N - 1
        if not (isinstance(u, torch.Tensor) and u.is_cuda and u.dtype == torch.float32 and u.is_contiguous()
                and u.dim() == 3 and tuple(u.shape[1:]) == (n, n)):
            raise ValueError(f"{name} must be a contiguous CUDA float32 tensor of shape (B, {n}, {n})")
        return ctypes.c_void_p(u.data_ptr())

    def forward(self, u, D: Sequence[float], out=None, stream=None):
        torch = _torch()
        out = torch.empty_like(u) if out is None else out
        Da, B = _darr(D)
        if B != u.shape[0]:
            raise ValueError("one D per field")
        nat.check(nat.lib().etd_sno_forward(self._h, self._field(u), Da, B, self._field(out, "out"),
                                            _stream_ptr(stream)), "etd_sno_forward")
        return out

    def train_step(self, u, D: Sequence[float], target, lr: float, stream=None) -> float:
        Da, B = _darr(D)
        loss = ctypes.c_double()
        nat.check(nat.lib().etd_sno_train_step(self._h, self._field(u), Da, self._field(target, "target"), B,
                                               ctypes.c_float(lr), ctypes.byref(loss), None, _stream_ptr(stream)),
                  "etd_sno_train_step")
        return loss.value

    def gradient(self, u, D: Sequence[float], target, stream=None) -> tuple:
        """(loss, gradient dict) without updating the parameters."""
        Da, B = _darr(D)
        loss = ctypes.c_double()
        flat = np.empty(self.nparam, dtype=np.float32)
        nat.check(nat.lib().etd_sno_train_step(self._h, self._field(u), Da, self._field(target, "target"), B,
                                               ctypes.c_float(0.0), ctypes.byref(loss),
                                               flat.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream)),
                  "etd_sno_train_step")
        return loss.value, unflatten(flat, self.C, self.M, self.L)

    def close(self):
        if getattr(self, "_h", None):
            nat.lib().etd_sno_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Parareal:
    """Parareal for B problems at N x N with coefficients D: `windows` windows of `window_steps`
    ETDRK2 steps of size tau; coarse propagator `sno` (None: one ETDRK2 step of window_steps * tau)."""

    def __init__(self, sno: Optional[Sno], N: int, D: Sequence[float], tau: float, window_steps: int, windows: int):
        Da, B = _darr(D)
        self.B, self.N, self.sno = B, int(N), sno
        h = ctypes.c_void_p()
        nat.check(nat.lib().etd_parareal_create(ctypes.byref(h), sno._h if sno is not None else None, self.N, B, Da,
                                                float(tau), int(window_steps), int(windows)), "etd_parareal_create")
        self._h = h

    def run(self, u0, max_iter: int, tol: float, fallback_tol: float = 1e-2, out=None, stream=None) -> tuple:
        torch = _torch()
        out = torch.empty_like(u0) if out is None else out
        st = nat.EtdPararealStats()
        nat.check(nat.lib().etd_parareal_run(self._h, ctypes.c_void_p(u0.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                             int(max_iter), float(tol), float(fallback_tol), ctypes.byref(st),
                                             _stream_ptr(stream)), "etd_parareal_run")
        return out, {"iterations": st.iterations, "fallbacks": st.fallbacks,
                     "correction": [st.correction[i] for i in range(st.iterations)]}

    def close(self):
        if getattr(self, "_h", None):
            nat.lib().etd_parareal_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
