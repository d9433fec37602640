"""Arithmetic identities the kernels rely on, checked with IEEE arithmetic on the host.

* Centre means (Sec. II-D): for integers |a|, b < 2^24 (exact floats), the float32 quotient equals
  the float64 quotient rounded to float32 (double rounding is innocuous for a division because
  53 >= 2 x 24 + 2), also after the exact scaling by 1/1024.
* Mask comparison (Eq. 17): for a float x and a double t, x < t exactly when x < t rounded up to
  a float.
"""
import numpy as np


def test_float_division_equals_rounded_double_division():
    rng = np.random.default_rng(3)
    n = 400000
    b = rng.integers(1, 1 << 24, n)
    a = rng.integers(-(1 << 24) + 1, 1 << 24, n)
    # quotients near float midpoints: a = b * (odd multiple of half a float ulp) rounded
    edge_b = rng.integers(1, 1 << 12, 2000)
    edge_a = (edge_b * 1000.5).astype(np.int64)
    a = np.concatenate([a, edge_a, [(1 << 24) - 1, -(1 << 24) + 1, 0, 1]])
    b = np.concatenate([b, edge_b, [3, 7, 5, (1 << 24) - 1]])
    f32 = np.float32(a) / np.float32(b)
    via64 = (np.float64(a) / np.float64(b)).astype(np.float32)
    assert np.array_equal(f32, via64)
    assert np.array_equal(f32 * np.float32(1.0 / 1024.0),
                          (np.float64(a) / np.float64(b) / 1024.0).astype(np.float32))


def _round_up_to_float(t):
    with np.errstate(over="ignore"):  # beyond the float range t rounds to infinity
        f = np.float32(t)
    return f if np.float64(f) >= t else np.nextafter(f, np.float32(np.inf))


def test_float_compare_against_threshold_rounded_up():
    rng = np.random.default_rng(4)
    ts = np.concatenate([rng.normal(16.0, 3.0, 300), [0.1, 1.0 / 3.0, -2.36, 1e-30, 3.5e38]])
    for t in ts:
        tf = _round_up_to_float(t)
        with np.errstate(over="ignore"):
            f = np.float32(t)
        xs = np.array([f, np.nextafter(f, np.float32(-np.inf)), np.nextafter(f, np.float32(np.inf)),
                       tf, np.nextafter(tf, np.float32(-np.inf)), np.float32(-np.inf),
                       np.float32(np.inf), np.float32(np.nan)], np.float32)
        assert np.array_equal(np.float64(xs) < t, xs < tf)
