"""The phi-function weights of the stage combinations (phi_k of Section 2.2 in eqs. (2.13)/(2.14)) as
the FFT pass kernels evaluate them per mode (etd_phi_weights runs the kernels' own device functions),
against 50-digit values of the closed forms phi_1(z) = (e^z - 1)/z, phi_2(z) = (e^z - 1 - z)/z^2
(Python's decimal module, so the check runs wherever the GPU does).

The grid spans zeta in [1e-8, 1e3] and every workload's range of zeta = tau D (mu_x + mu_y [+ mu_z]):
1e-5 to 13 at 1024^2 (tau D = 5e-7), 3e-4 to 24 at 256^3 (tau D = 1e-5), up to 10 at 64^2, with points on
both sides of the switch between series and closed form (zeta = 1, c2 zeta = 1). Each weight is compared
with the exact value at the zeta the kernels hold (zeta rounded to the plan's type; E = e^{-zeta} and
e^{-c2 zeta} rounded likewise, as the per-axis tables and their products are). Bounds: FP32 8 ulp
relative (4.8e-7), FP64 64 ulp (1.4e-14)."""
from decimal import Decimal, getcontext
import ctypes

import numpy as np
import pytest

from paper_2209_11922_gb300 import _native as nat

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

getcontext().prec = 50


def _exact(z: float, c2: float):
    """phi_1(-z), phi_2(-z), c2 phi_1(-c2 z) to 50 digits for z > 0 (z is taken exactly as given)."""
    Z, C2 = Decimal(z), Decimal(c2)
    if Z == 0:
        return 1.0, 0.5, c2
    e = (-Z).exp()
    p1 = (1 - e) / Z
    p2 = (e - 1 + Z) / (Z * Z)
    zc = C2 * Z
    p1c = C2 * (1 - (-zc).exp()) / zc
    return float(p1), float(p2), float(p1c)


def _grid():
    z = np.concatenate([np.logspace(-8, 3, 600), [0.0, 0.999, 0.9999999, 1.0, 1.0000001, 1.001, 1.999, 1.9999999,
                                                   2.0, 2.0000001, 2.001, 5e-7 * 19.74, 12.6, 1e-5 * 29.6, 23.6]])
    return np.unique(z)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_phi_weights_match_closed_forms(dtype):
    L = nat.lib()
    c2 = 0.5
    npdt = np.float32 if dtype == "f32" else np.float64
    z = _grid().astype(npdt).astype(np.float64)          # the zeta the kernels hold
    E = np.exp(-z).astype(npdt).astype(np.float64)
    Ec = np.exp(-c2 * z).astype(npdt).astype(np.float64)
    n = len(z)
    out = np.zeros(3 * n)
    P = ctypes.POINTER(ctypes.c_double)
    st = L.etd_phi_weights(nat.ETD_F32 if dtype == "f32" else nat.ETD_F64, n, z.ctypes.data_as(P),
                           E.ctypes.data_as(P), Ec.ctypes.data_as(P), c2, out.ctypes.data_as(P))
    nat.check(st, "etd_phi_weights")
    got = out.reshape(n, 3)
    ref = np.array([_exact(float(v), c2) for v in z])
    rel = np.abs(got - ref) / np.abs(ref)
    eps = np.finfo(npdt).eps / 2
    bound = (8 if dtype == "f32" else 64) * eps
    worst = np.unravel_index(rel.argmax(), rel.shape)
    assert rel.max() <= bound, (dtype, float(rel.max()), float(z[worst[0]]), worst[1], bound)
