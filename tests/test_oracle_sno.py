"""Pins of the spectral-neural-operator oracle and its Parareal iteration (no GPU)."""
import numpy as np
import pytest

from oracle import sno
from oracle import transforms as otr
from paper_2209_11922_gb300 import inputs

TINY = inputs.SnoWorkload("tiny", N=8, C=3, M=3, L=2)


def _params(w: inputs.SnoWorkload, scale_q=1.0) -> sno.Params:
    d = w.init_weights()
    P = sno.Params(*[np.array(d[n], dtype=np.float64) for n in sno.Params.NAMES])
    P.Wq = P.Wq * scale_q
    P.bl = P.bl + 0.1
    P.bp = P.bp - 0.05
    P.bq = np.array(0.02)
    return P


def _batch(w, B=2):
    u = np.stack([w.u0(i) for i in range(B)])
    D = np.array([w.D(i) for i in range(B)])
    return u, D


def test_mode_matrix_is_the_leading_rows_of_the_orthonormal_sine_matrix():
    S = sno.mode_matrix(16, 5)
    assert np.allclose(S @ S.T, np.eye(5), atol=1e-14)
    y = np.arange(1, 16)
    assert np.allclose(S[2], np.sqrt(2 / 16) * np.sin(3 * y * np.pi / 16), atol=1e-15)
    assert np.allclose(S, otr.sine_matrix(16)[:5])


def test_gelu_closed_forms():
    assert sno.gelu(np.array(0.0)) == 0.0
    assert abs(sno.gelu(np.array(8.0)) - 8.0) < 1e-12 and abs(sno.gelu(np.array(-8.0))) < 1e-12
    assert abs(sno.gelu_grad(np.array(0.0)) - 0.5) < 1e-15
    z = np.linspace(-3, 3, 13)
    fd = (sno.gelu(z + 1e-6) - sno.gelu(z - 1e-6)) / 2e-6
    assert np.allclose(sno.gelu_grad(z), fd, atol=1e-8)


def test_bf16_rounding_is_nearest_even_to_8_significant_bits():
    assert sno.bf16(1.0 + 2.0 ** -8) == 1.0                 # tie -> even
    assert sno.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie -> even (up)
    assert sno.bf16(1.0 + 2.0 ** -7) == 1.0 + 2.0 ** -7
    x = np.random.default_rng(1).normal(size=1000)
    assert np.max(np.abs(sno.bf16(x) - x) / np.abs(x)) <= 2.0 ** -8


def test_input_feature_maps_the_training_range_to_plus_minus_half():
    assert np.allclose(sno.feature([1e-4, 1e-3, 1e-2]), [-0.5, 0.0, 0.5])


@pytest.mark.parametrize("name", sno.Params.NAMES)
def test_backward_matches_central_differences(name):
    """Every parameter's gradient against central differences of the loss (bf16 rounding off, so
    that the loss is smooth in the mix weights)."""
    w = TINY
    P = _params(w, scale_q=5.0)
    u, D = _batch(w)
    target = u + 0.05 * np.stack([w.u0(10 + i) for i in range(2)])
    uh, cache = sno.forward(P, u, D, w.N, rounding=False)
    g = sno.backward(P, cache, uh, target, w.N)
    arr = getattr(P, name)
    ga = getattr(g, name)
    flat = arr.reshape(-1)
    idx = np.unique(np.linspace(0, flat.size - 1, min(flat.size, 12)).astype(int))
    for i in idx:
        eps = 1e-6
        old = flat[i]
        flat[i] = old + eps
        lp = sno.loss(sno.forward(P, u, D, w.N, rounding=False)[0], target)
        flat[i] = old - eps
        lm = sno.loss(sno.forward(P, u, D, w.N, rounding=False)[0], target)
        flat[i] = old
        fd = (lp - lm) / (2 * eps)
        an = ga.reshape(-1)[i]
        assert abs(fd - an) <= 1e-7 + 1e-5 * abs(fd), (name, i, fd, an)


def test_rounded_forward_stays_within_bf16_error_of_the_exact_one():
    w = TINY
    P = _params(w)
    u, D = _batch(w)
    a = sno.forward(P, u, D, w.N, rounding=True)[0] - u
    b = sno.forward(P, u, D, w.N, rounding=False)[0] - u
    assert np.linalg.norm(a - b) <= 2.0 ** -7 * np.linalg.norm(b)
    assert np.linalg.norm(a - b) > 0


def test_adam_first_step_moves_each_weight_by_lr():
    P = _params(TINY)
    g = sno.zeros_like(P)
    g.Wp = np.random.default_rng(2).normal(size=P.Wp.shape)
    before = P.Wp.copy()
    opt = sno.Adam(lr=1e-2, eps=1e-30)
    opt.step(P, g)
    assert np.allclose(P.Wp - before, -1e-2 * np.sign(g.Wp), atol=1e-15)
    assert np.array_equal(P.Wm, _params(TINY).Wm)   # zero gradient, zero step


def test_parareal_is_exact_on_the_first_k_windows_after_k_iterations():
    fine = lambda x: 0.9 * x + 0.1 * np.sin(x)
    coarse = lambda x: 0.8 * x
    u0 = np.array([0.7, -0.3])
    its = sno.parareal(u0, 4, fine, coarse, 4)
    exact = [u0]
    for _ in range(4):
        exact.append(fine(exact[-1]))
    for k, U in enumerate(its):
        for n in range(k + 1):
            assert np.allclose(U[n], exact[n], atol=1e-15), (k, n)
    assert np.allclose(its[4][4], exact[4], atol=1e-15)
    assert not np.allclose(its[1][4], exact[4])


def test_parareal_with_the_fine_propagator_as_coarse_converges_in_one_iteration():
    fine = lambda x: np.cos(x)
    its = sno.parareal(np.array([0.2]), 3, fine, fine, 1)
    assert np.allclose(its[1][3], fine(fine(fine(np.array([0.2])))), atol=1e-15)
