"""etd_monitor_noalloc: the monitors for callers that cannot allocate GPU memory (for example code
running under a framework that owns every allocation, or a real-time loop where allocation is not
allowed). It keeps its partial sums in a fixed array inside the library instead of memory it
allocates; this test checks it against etd_monitor (which uses a plan's scratch) on two calls in a
row, so a second call cannot pass by reading what the first left in the shared array.
This file is collected last so that a run stopping at the first failure has run every other test."""
import ctypes

import numpy as np
import pytest

from paper_2209_11922_gb300 import _native as nat
from paper_2209_11922_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(N, h, D, dtype, u):
    L = nat.lib()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")     # one etd_monitors (32 bytes)
    Na = (ctypes.c_int64 * 3)(*(list(N) + [1] * (3 - len(N))))
    ha = (ctypes.c_double * 3)(*(list(h) + [1.0] * (3 - len(N))))
    st = L.etd_monitor_noalloc(len(N), Na, ha, D, nat.ETD_F32 if u.dtype == torch.float32 else nat.ETD_F64,
                               ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    nat.check(st, "etd_monitor_noalloc")
    torch.cuda.synchronize()
    vals = out.cpu().numpy()
    return {"mass": vals[0], "energy": vals[1], "maxabs": vals[2],
            "nonfinite": int(np.frombuffer(vals[3:4].tobytes(), dtype=np.int64)[0])}


@pytest.mark.parametrize("N,dtype", [((64, 48), "f64"), ((256, 256, 256), "f32")])
def test_noalloc_matches_plan_monitor_on_two_calls(N, dtype):
    from paper_2209_11922_gb300.etd import Plan
    h = tuple(1.0 / n for n in N)
    D = 1e-3
    shape = tuple(n - 1 for n in reversed(N))
    with Plan(N, D, 0.01, dtype=dtype) as pl:
        for seed, amp in ((31, 0.9), (32, 1.3)):          # two calls in a row, different fields
            U = inputs.uniform_field(shape, -amp, amp, seed=seed)
            u = torch.from_numpy(U.astype(np.float32 if dtype == "f32" else np.float64)).cuda()
            ref = pl.monitor(u)
            got = _noalloc(N, h, D, dtype, u)
            for k in ("mass", "energy", "maxabs"):
                assert got[k] == pytest.approx(ref[k], rel=1e-12), (k, seed)
            assert got["nonfinite"] == ref["nonfinite"] == 0


def test_noalloc_counts_nonfinite_and_rejects_oversize():
    U = inputs.uniform_field((31, 31), -1, 1, seed=3)
    U[4, 5] = np.inf
    u = torch.from_numpy(U).cuda()
    assert _noalloc((32, 32), (1 / 32, 1 / 32), 0.1, "f64", u)["nonfinite"] == 1
    L = nat.lib()
    Na = (ctypes.c_int64 * 3)(1024, 1024, 64)             # 1023*1023*63 unknowns > the maximum
    ha = (ctypes.c_double * 3)(1e-3, 1e-3, 1e-2)
    st = L.etd_monitor_noalloc(3, Na, ha, 0.1, nat.ETD_F32, ctypes.c_void_p(u.data_ptr()),
                               ctypes.c_void_p(u.data_ptr()), None)
    assert st == nat.ETD_ERR_INVALID_ARG and b"maximum" in L.etd_last_error()
