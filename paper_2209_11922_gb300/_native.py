"""ctypes declarations of the C ABI in include/etd.h (argument marshalling only).

The shared library is built in-tree by ``paper_2209_11922_gb300.build`` (``__graft_entry__.build()``).
Loading fails loudly when it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libetd_gb300.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "etd.h")
HEADERS = [HEADER, os.path.join(os.path.dirname(HERE), "include", "etd_sno.h")]

c_int, c_double, c_int64, c_void_p, c_char_p = (ctypes.c_int, ctypes.c_double, ctypes.c_int64,
                                                ctypes.c_void_p, ctypes.c_char_p)

ETD_OK, ETD_ERR_INVALID_ARG, ETD_ERR_UNSUPPORTED, ETD_ERR_CUDA, ETD_ERR_OOM, ETD_ERR_NONFINITE, ETD_ERR_TIMEOUT = range(7)
ETD_DEBUG_STALL_FIRST_GEMM_PASS = 0x5A11
ETD_DEBUG_BATCH_SERIAL = 0x5A12
ETD_DEBUG_BATCH_PARALLEL = 0x5A13
ETD_F64, ETD_F32 = 0, 1
ETD_ROUTE_AUTO, ETD_ROUTE_FFT, ETD_ROUTE_FFT_HALF, ETD_ROUTE_GEMM_TF32, ETD_ROUTE_GEMM_BF16X3, ETD_ROUTE_FFT_SPLIT = 0, 1, 2, 3, 4, 5
ETD_BC_DIRICHLET, ETD_BC_PERIODIC = 0, 1
ETD_NUM_PASS_KINDS = 9


class EtdPararealStats(ctypes.Structure):
    _fields_ = [("iterations", c_int), ("fallbacks", c_int), ("correction", c_double * 32)]


class EtdOptions(ctypes.Structure):
    _fields_ = [("dtype", c_int), ("route", c_int), ("c2", c_double), ("flin", c_double), ("fcub", c_double),
                ("debug", c_int), ("bc", c_int), ("flog", c_double)]


class EtdMonitors(ctypes.Structure):
    _fields_ = [("mass", c_double), ("energy", c_double), ("maxabs", c_double), ("nonfinite", c_int64)]


class EtdPlanInfo(ctypes.Structure):
    _fields_ = [("ndim", c_int), ("N", c_int64 * 3), ("unknowns", c_int64), ("workspace_bytes", c_int64),
                ("kernels_per_step", c_int), ("bytes_per_step", c_double), ("dtype", c_int), ("scheme", c_int)]


# int (*etd_boundary_fn)(double t, double* g, double* gdot, void* ctx)
BOUNDARY_FN = ctypes.CFUNCTYPE(c_int, c_double, ctypes.POINTER(c_double), ctypes.POINTER(c_double), c_void_p)

_SIGS = {
    "etd_options_default": (c_int, [ctypes.POINTER(EtdOptions)]),
    "etd_plan_create": (c_int, [ctypes.POINTER(c_void_p), c_int, ctypes.POINTER(c_int64),
                                ctypes.POINTER(c_double), c_double, c_double, c_int, ctypes.POINTER(EtdOptions)]),
    "etd_run": (c_int, [c_void_p, c_void_p, c_int64, c_void_p]),
    "etd_step": (c_int, [c_void_p, c_void_p, c_void_p]),
    "etd_run_from": (c_int, [c_void_p, c_void_p, c_int64, c_double, c_void_p]),
    "etd_set_source": (c_int, [c_void_p, c_double, c_double, ctypes.POINTER(c_double), ctypes.POINTER(c_double),
                               ctypes.POINTER(c_double)]),
    "etd_set_boundary": (c_int, [c_void_p, BOUNDARY_FN, c_void_p]),
    "etd_boundary_count": (c_int, [c_void_p, ctypes.POINTER(c_int64)]),
    "etd_run_host": (c_int, [c_void_p, c_void_p, c_int64, c_void_p]),
    "etd_apply_dst": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "etd_monitor": (c_int, [c_void_p, c_void_p, ctypes.POINTER(EtdMonitors), c_void_p]),
    "etd_run_profiled": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, ctypes.POINTER(c_double),
                                 ctypes.POINTER(c_int64)]),
    "etd_get_plan_info": (c_int, [c_void_p, ctypes.POINTER(EtdPlanInfo)]),
    "etd_pass_kind_name": (c_char_p, [c_int]),
    "etd_destroy": (c_int, [c_void_p]),
    "etd_batch_create": (c_int, [ctypes.POINTER(c_void_p), c_int, ctypes.POINTER(c_int64), ctypes.POINTER(c_double),
                                 ctypes.POINTER(c_double), c_double, c_int, ctypes.POINTER(EtdOptions)]),
    "etd_batch_run": (c_int, [c_void_p, ctypes.POINTER(c_void_p), c_int64, c_void_p]),
    "etd_batch_info": (c_int, [c_void_p, ctypes.POINTER(c_int64), ctypes.POINTER(c_int), ctypes.POINTER(c_int), c_int]),
    "etd_batch_schedule": (c_int, [c_void_p, ctypes.POINTER(c_int), ctypes.POINTER(c_double), ctypes.POINTER(c_double)]),
    "etd_batch_destroy": (c_int, [c_void_p]),
    "etd_monitor_noalloc": (c_int, [c_int, ctypes.POINTER(c_int64), ctypes.POINTER(c_double), c_double, c_int,
                                    c_void_p, c_void_p, c_void_p]),
    "etd_phi_weights": (c_int, [c_int, c_int64, ctypes.POINTER(c_double), ctypes.POINTER(c_double),
                                ctypes.POINTER(c_double), c_double, ctypes.POINTER(c_double)]),
    "etd_sno_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_int, c_int, c_int, c_int]),
    "etd_sno_param_count": (c_int64, [c_void_p]),
    "etd_sno_set_params": (c_int, [c_void_p, c_void_p]),
    "etd_sno_get_params": (c_int, [c_void_p, c_void_p]),
    "etd_sno_forward": (c_int, [c_void_p, c_void_p, ctypes.POINTER(c_double), c_int, c_void_p, c_void_p]),
    "etd_sno_train_step": (c_int, [c_void_p, c_void_p, ctypes.POINTER(c_double), c_void_p, c_int, ctypes.c_float,
                                   ctypes.POINTER(c_double), c_void_p, c_void_p]),
    "etd_sno_destroy": (c_int, [c_void_p]),
    "etd_parareal_create": (c_int, [ctypes.POINTER(c_void_p), c_void_p, c_int, c_int, ctypes.POINTER(c_double),
                                    c_double, c_int, c_int]),
    "etd_parareal_run": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_double, c_double, c_void_p, c_void_p]),
    "etd_parareal_destroy": (c_int, [c_void_p]),
    "etd_status_string": (c_char_p, [c_int]),
    "etd_last_error": (c_char_p, []),
}

_lib = None


def header_functions() -> list:
    """Names of the functions declared in include/etd.h and include/etd_sno.h."""
    text = "\n".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(etd_[a-z_0-9]+)\s*\(",
                                 text, flags=re.M)))


def lib() -> ctypes.CDLL:
    """Load the library once; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing; run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


class EtdError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = lib()
        self.status = status
        msg = L.etd_status_string(status).decode()
        detail = L.etd_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}): {detail}")


def check(status: int, where: str) -> None:
    if status != ETD_OK:
        raise EtdError(status, where)
