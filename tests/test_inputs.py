"""The seeded generator against the published SplitMix64 definition and its known first outputs."""
import numpy as np
import pytest

from paper_2209_11922_gb300 import inputs


def _splitmix64_scalar(seed, n):
    """Straight transcription of the published recurrence with Python integers."""
    m = (1 << 64) - 1
    x, out = seed & m, []
    for _ in range(n):
        x = (x + 0x9E3779B97F4A7C15) & m
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
        out.append(z ^ (z >> 31))
    return out


def test_known_first_outputs_for_seed_zero():
    got = [int(v) for v in inputs.splitmix64(0, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_vectorised_stream_matches_recurrence():
    for seed in (1, 20220923, (1 << 64) - 5):
        np.testing.assert_array_equal(inputs.splitmix64(seed, 50).astype(object),
                                      np.array(_splitmix64_scalar(seed, 50), dtype=object))
    # counter-based: an offset continues the same stream
    np.testing.assert_array_equal(inputs.splitmix64(9, 10, offset=40), inputs.splitmix64(9, 50)[40:])


def test_uniform_field_range_and_shape():
    u = inputs.uniform_field((7, 9), -0.9, 0.9, seed=3)
    assert u.shape == (7, 9) and u.dtype == np.float64
    assert u.min() >= -0.9 and u.max() < 0.9
    w = inputs.AC2D_1024
    assert inputs.interior_shape(w.N) == (1023, 1023) and w.unknowns == 1023 * 1023


def test_field_shapes_and_workload_sizes():
    from paper_2209_11922_gb300 import inputs
    assert inputs.field_shape((8, 6), "dirichlet") == (5, 7)
    assert inputs.field_shape((8, 6), "periodic") == (6, 8)
    assert inputs.field_shape((8, 6, 4), "periodic") == (4, 6, 8)
    with pytest.raises(ValueError):
        inputs.field_shape((8, 6), "neumann")
    w = inputs.GC3D_128
    assert w.bc == "periodic" and w.shape == (128, 128, 128) and w.unknowns == 128 ** 3
    assert (w.flin, w.fcub, w.flog) == (1.6, 0.0, -0.8) and w.D == pytest.approx(0.01 ** 2)
    assert w.tau * w.nsteps == pytest.approx(20.0)       # Example 5.3: T = 20, N_T = 2048
    u = w.u0()
    assert u.shape == w.shape and u.min() >= -0.9 and u.max() < 0.9
    a = inputs.AC2D_1024
    assert a.bc == "dirichlet" and a.unknowns == 1023 ** 2 and a.u0().shape == (1023, 1023)
