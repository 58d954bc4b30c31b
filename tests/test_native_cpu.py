"""Host-side checks of the C-ABI library that need no GPU: it loads, exports every function that
include/etd.h declares, and rejects invalid arguments before touching the device."""
import ctypes

import numpy as np
import pytest

from paper_2209_11922_gb300 import _native as nat


@pytest.fixture(scope="module")
def L():
    try:
        return nat.lib()
    except RuntimeError as e:  # the library is built by __graft_entry__.build()
        pytest.fail(str(e))


def test_library_exports_every_declared_function(L):
    names = nat.header_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n
    assert set(nat._SIGS) <= set(names)


def _create(L, ndim, N, h, D=0.1, tau=0.01, scheme=2, opt=None):
    Na = (ctypes.c_int64 * 3)(*N)
    ha = (ctypes.c_double * 3)(*h)
    p = ctypes.c_void_p()
    return L.etd_plan_create(ctypes.byref(p), ndim, Na, ha, D, tau, scheme, opt), p


@pytest.mark.parametrize("case", [
    dict(ndim=1), dict(ndim=4), dict(N=(1, 8, 1)), dict(N=(7, 8, 1)), dict(h=(0.0, 0.1, 1)),
    dict(h=(-1.0, 0.1, 1)), dict(D=0.0), dict(D=float("nan")), dict(tau=-1.0), dict(scheme=3),
    dict(tau=float("inf")),
])
def test_invalid_arguments_are_rejected_on_the_host(L, case):
    args = dict(ndim=2, N=(8, 8, 1), h=(0.125, 0.125, 1.0), D=0.1, tau=0.01, scheme=2)
    args.update(case)
    st, p = _create(L, args["ndim"], args["N"], args["h"], args["D"], args["tau"], args["scheme"])
    assert st == nat.ETD_ERR_INVALID_ARG and not p.value
    assert L.etd_last_error()  # a detail string is set


@pytest.mark.parametrize("c2", [0.0, 1.5, float("nan")])
def test_invalid_c2_rejected(L, c2):
    opt = nat.EtdOptions()
    L.etd_options_default(ctypes.byref(opt))
    opt.c2 = c2
    st, _ = _create(L, 2, (8, 8, 1), (0.125, 0.125, 1.0), opt=ctypes.byref(opt))
    assert st == nat.ETD_ERR_INVALID_ARG


def test_unsupported_axis_length(L):
    st, _ = _create(L, 2, (10, 8, 1), (0.1, 0.125, 1.0))
    assert st == nat.ETD_ERR_UNSUPPORTED
    st, _ = _create(L, 3, (8, 8, 4096), (0.1, 0.125, 1.0))
    assert st == nat.ETD_ERR_UNSUPPORTED


def test_null_arguments(L):
    assert L.etd_run(None, None, 1, None) == nat.ETD_ERR_INVALID_ARG
    assert L.etd_monitor(None, None, None, None) == nat.ETD_ERR_INVALID_ARG
    assert L.etd_destroy(None) == nat.ETD_OK
    assert L.etd_options_default(None) == nat.ETD_ERR_INVALID_ARG


def test_defaults_and_names(L):
    opt = nat.EtdOptions()
    assert L.etd_options_default(ctypes.byref(opt)) == nat.ETD_OK
    assert (opt.dtype, opt.c2, opt.flin, opt.fcub) == (nat.ETD_F64, 0.5, 1.0, -1.0)
    assert (opt.bc, opt.flog, opt.debug) == (nat.ETD_BC_DIRICHLET, 0.0, 0)
    assert L.etd_status_string(nat.ETD_ERR_NONFINITE) == b"non-finite values"
    assert [L.etd_pass_kind_name(k) for k in range(nat.ETD_NUM_PASS_KINDS)][1] == b"x_react"
    assert L.etd_pass_kind_name(99) is None


def test_batch_arguments_rejected_on_the_host(L):
    p = ctypes.c_void_p()
    N = (ctypes.c_int64 * 4)(64, 64, 63, 64)
    h = (ctypes.c_double * 4)(1 / 64, 1 / 64, 1 / 63, 1 / 64)
    D = (ctypes.c_double * 2)(1e-3, 1e-3)
    assert L.etd_batch_create(ctypes.byref(p), 0, N, h, D, 0.01, 2, None) == nat.ETD_ERR_INVALID_ARG
    assert L.etd_batch_create(ctypes.byref(p), 2, N, h, D, 0.01, 2, None) == nat.ETD_ERR_INVALID_ARG  # odd N
    N2 = (ctypes.c_int64 * 4)(64, 64, 80, 64)
    assert L.etd_batch_create(ctypes.byref(p), 2, N2, h, D, 0.01, 2, None) == nat.ETD_ERR_UNSUPPORTED
    D2 = (ctypes.c_double * 2)(1e-3, -1.0)
    N3 = (ctypes.c_int64 * 4)(64, 64, 64, 64)
    assert L.etd_batch_create(ctypes.byref(p), 2, N3, h, D2, 0.01, 2, None) == nat.ETD_ERR_INVALID_ARG
    assert L.etd_batch_run(None, None, 1, None) == nat.ETD_ERR_INVALID_ARG
    assert L.etd_batch_destroy(None) == nat.ETD_OK
    assert L.etd_batch_schedule(None, None, None, None) == nat.ETD_ERR_INVALID_ARG


def _opts(L, dtype=None, route=None):
    opt = nat.EtdOptions()
    L.etd_options_default(ctypes.byref(opt))
    if dtype is not None:
        opt.dtype = dtype
    if route is not None:
        opt.route = route
    return opt


def test_gemm_route_arguments_rejected_on_the_host(L):
    for route in (nat.ETD_ROUTE_GEMM_TF32, nat.ETD_ROUTE_GEMM_BF16X3):
        # FP64 plans have no tensor-core route
        opt = _opts(L, nat.ETD_F64, route)
        st, p = _create(L, 2, (64, 64, 1), (1 / 64, 1 / 64, 1.0), opt=ctypes.byref(opt))
        assert st == nat.ETD_ERR_INVALID_ARG and not p.value
        # axis lengths must be multiples of 32 (48 has FFT kernels, but no GEMM tiling)
        opt = _opts(L, nat.ETD_F32, route)
        st, p = _create(L, 2, (64, 48, 1), (1 / 64, 1 / 48, 1.0), opt=ctypes.byref(opt))
        assert st == nat.ETD_ERR_UNSUPPORTED and not p.value
        # batches run the FFT routes only
        b = ctypes.c_void_p()
        N = (ctypes.c_int64 * 2)(64, 64)
        h = (ctypes.c_double * 2)(1 / 64, 1 / 64)
        D = (ctypes.c_double * 1)(1e-3)
        assert L.etd_batch_create(ctypes.byref(b), 1, N, h, D, 0.01, 2, ctypes.byref(opt)) == nat.ETD_ERR_UNSUPPORTED
    opt = _opts(L, nat.ETD_F32, 7)
    st, _ = _create(L, 2, (64, 64, 1), (1 / 64, 1 / 64, 1.0), opt=ctypes.byref(opt))
    assert st == nat.ETD_ERR_INVALID_ARG
    assert L.etd_status_string(nat.ETD_ERR_TIMEOUT) == b"a device wait ran out"


def test_sno_and_parareal_arguments_rejected_on_the_host(L):
    p = ctypes.c_void_p()
    for args in [(7, 8, 4, 2, 4), (64, 0, 4, 2, 4), (64, 8, 64, 2, 4), (64, 8, 4, 0, 4), (64, 8, 4, 2, 0),
                 (64, 300, 4, 2, 4), (64, 32, 4, 2, 4096)]:
        assert L.etd_sno_create(ctypes.byref(p), *args) == nat.ETD_ERR_INVALID_ARG, args
        assert not p.value
    assert L.etd_sno_create(None, 64, 8, 4, 2, 4) == nat.ETD_ERR_INVALID_ARG
    assert L.etd_sno_param_count(None) == 0
    assert L.etd_sno_destroy(None) == nat.ETD_OK
    D = (ctypes.c_double * 2)(1e-3, 1e-3)
    assert L.etd_parareal_create(ctypes.byref(p), None, 64, 0, D, 0.01, 50, 4) == nat.ETD_ERR_INVALID_ARG
    assert L.etd_parareal_create(ctypes.byref(p), None, 64, 2, D, 0.01, 50, 0) == nat.ETD_ERR_INVALID_ARG
    assert L.etd_parareal_create(ctypes.byref(p), None, 64, 2, D, -1.0, 50, 4) == nat.ETD_ERR_INVALID_ARG
    assert L.etd_parareal_run(None, None, None, 1, 0.0, 0.0, None, None) == nat.ETD_ERR_INVALID_ARG
    assert L.etd_parareal_destroy(None) == nat.ETD_OK


def test_sno_parameter_layout_round_trips():
    """The flat parameter layout of the binding matches the documented order and sizes."""
    import numpy as np

    from paper_2209_11922_gb300 import inputs, sno
    w = inputs.SnoWorkload("t", N=16, C=3, M=2, L=2)
    P = w.init_weights()
    flat = sno.flatten(P)
    assert flat.size == 2 * 3 + 3 + 2 * 2 * 2 * 3 * 3 + 2 * 3 * 3 + 2 * 3 + 3 + 1
    back = sno.unflatten(flat, 3, 2, 2)
    for k in sno.PARAM_NAMES:
        assert np.allclose(back[k], np.asarray(P[k], dtype=np.float32)), k


def test_periodic_and_log_reaction_arguments_rejected_on_the_host(L):
    opt = _opts(L, nat.ETD_F32)
    opt.bc = 5
    st, p = _create(L, 2, (64, 64, 1), (1 / 64, 1 / 64, 1.0), opt=ctypes.byref(opt))
    assert st == nat.ETD_ERR_INVALID_ARG and not p.value
    opt = _opts(L, nat.ETD_F32)
    opt.flog = float("nan")
    st, p = _create(L, 2, (64, 64, 1), (1 / 64, 1 / 64, 1.0), opt=ctypes.byref(opt))
    assert st == nat.ETD_ERR_INVALID_ARG and not p.value
    for route in (nat.ETD_ROUTE_GEMM_TF32, nat.ETD_ROUTE_GEMM_BF16X3):
        opt = _opts(L, nat.ETD_F32, route)
        opt.bc = nat.ETD_BC_PERIODIC
        st, p = _create(L, 2, (64, 48, 1), (1 / 64, 1 / 48, 1.0), opt=ctypes.byref(opt))
        assert st == nat.ETD_ERR_UNSUPPORTED and not p.value     # multiples of 32 on these routes too
    opt = _opts(L, nat.ETD_F32)
    opt.flog = -0.8                     # the artanh term: periodic plans and GEMM routes only
    st, p = _create(L, 2, (64, 64, 1), (1 / 64, 1 / 64, 1.0), opt=ctypes.byref(opt))
    assert st == nat.ETD_ERR_UNSUPPORTED and not p.value
    opt = _opts(L, nat.ETD_F32)
    opt.bc = nat.ETD_BC_PERIODIC
    st, p = _create(L, 2, (64, 80, 1), (1 / 64, 1 / 80, 1.0), opt=ctypes.byref(opt))
    assert st == nat.ETD_ERR_UNSUPPORTED and not p.value     # no kernel for 80
    b = ctypes.c_void_p()
    N = (ctypes.c_int64 * 2)(64, 64)
    h = (ctypes.c_double * 2)(1 / 64, 1 / 64)
    D = (ctypes.c_double * 1)(1e-3)
    opt = _opts(L, nat.ETD_F32)
    opt.flog = -0.8                     # Dirichlet batches take the polynomial reaction only
    assert L.etd_batch_create(ctypes.byref(b), 1, N, h, D, 0.01, 2, ctypes.byref(opt)) == nat.ETD_ERR_UNSUPPORTED
    opt.bc = 7
    assert L.etd_batch_create(ctypes.byref(b), 1, N, h, D, 0.01, 2, ctypes.byref(opt)) == nat.ETD_ERR_INVALID_ARG


def test_boundary_arguments_rejected_on_the_host(L):
    n = ctypes.c_int64()
    assert L.etd_boundary_count(None, ctypes.byref(n)) == nat.ETD_ERR_INVALID_ARG
    assert L.etd_set_boundary(None, nat.BOUNDARY_FN(), None) == nat.ETD_ERR_INVALID_ARG
    assert L.etd_pass_kind_name(8) == b"boundary"


@pytest.mark.parametrize("N", [(4, 6), (5, 3, 4)])
def test_boundary_layout_matches_the_header(N):
    """Plan.boundary_nodes() enumerates the faces in the order etd.h documents (x = 0, x = L_x, y = 0,
    y = L_y, z = 0, z = L_z; all nodes of each face, x fastest) and matches etd_boundary_count's size."""
    from paper_2209_11922_gb300.etd import Plan
    pl = object.__new__(Plan)
    pl.N, pl.ndim = tuple(N), len(N)
    got = np.stack(pl.boundary_nodes(), axis=1)
    want = []
    if len(N) == 2:
        Nx, Ny = N
        want += [(0, j) for j in range(Ny + 1)] + [(Nx, j) for j in range(Ny + 1)]
        want += [(i, 0) for i in range(Nx + 1)] + [(i, Ny) for i in range(Nx + 1)]
        count = 2 * (Ny + 1) + 2 * (Nx + 1)
    else:
        Nx, Ny, Nz = N
        for v in (0, Nx):
            want += [(v, j, k) for k in range(Nz + 1) for j in range(Ny + 1)]
        for v in (0, Ny):
            want += [(i, v, k) for k in range(Nz + 1) for i in range(Nx + 1)]
        for v in (0, Nz):
            want += [(i, j, v) for j in range(Ny + 1) for i in range(Nx + 1)]
        count = 2 * (Nz + 1) * (Ny + 1) + 2 * (Nz + 1) * (Nx + 1) + 2 * (Ny + 1) * (Nx + 1)
    assert got.shape[0] == count
    assert [tuple(r) for r in got] == want


@pytest.mark.parametrize("N", [(2 ** 21 + 1, 2 ** 21 + 1, 2 ** 21 + 1), (2 ** 30, 2 ** 30, 2), (6000, 6000, 2)])
def test_noalloc_monitor_rejects_oversize_without_overflow(L, N):
    """The size check of etd_monitor_noalloc runs axis by axis before each multiply: three axes of
    2^21 unknowns (2^63 in total, which wraps a 64-bit product) are rejected like any field above
    the maximum, on the host, before any device work."""
    Na = (ctypes.c_int64 * 3)(*N)
    ha = (ctypes.c_double * 3)(1e-3, 1e-3, 1e-3)
    dummy = ctypes.c_void_p(256)   # never dereferenced: the call fails in its argument checks
    st = L.etd_monitor_noalloc(3, Na, ha, 0.1, nat.ETD_F32, dummy, dummy, None)
    assert st == nat.ETD_ERR_INVALID_ARG and b"maximum" in L.etd_last_error()


def test_phi_weights_arguments_rejected_on_the_host(L):
    arr = (ctypes.c_double * 3)(0.1, 1.0, 2.0)
    out = (ctypes.c_double * 9)()
    assert L.etd_phi_weights(7, 3, arr, arr, arr, 0.5, out) == nat.ETD_ERR_INVALID_ARG
    assert L.etd_phi_weights(nat.ETD_F32, -1, arr, arr, arr, 0.5, out) == nat.ETD_ERR_INVALID_ARG
    assert L.etd_phi_weights(nat.ETD_F32, 3, None, arr, arr, 0.5, out) == nat.ETD_ERR_INVALID_ARG
    assert L.etd_phi_weights(nat.ETD_F32, 3, arr, arr, arr, 1.5, out) == nat.ETD_ERR_INVALID_ARG
    bad = (ctypes.c_double * 3)(0.1, -1.0, 2.0)
    assert L.etd_phi_weights(nat.ETD_F64, 3, bad, arr, arr, 0.5, out) == nat.ETD_ERR_INVALID_ARG
    assert L.etd_phi_weights(nat.ETD_F64, 0, None, None, None, 0.5, None) == nat.ETD_OK
