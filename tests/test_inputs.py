"""The seeded generator against the published SplitMix64 definition and its known first outputs."""
import numpy as np

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
