"""Arithmetic identities the kernels rely on, checked with IEEE arithmetic on the host.

* Centre means (Sec. II-D): for integers |a|, b < 2^24 (exact floats), the float32 quotient equals
  the float64 quotient rounded to float32 (double rounding is innocuous for a division because
  53 >= 2 x 24 + 2), also after the exact scaling by 1/1024.
* Mask comparison (Eq. 17): for a float x and a double t, x < t exactly when x < t rounded up to
  a float.
* Fixed-point values rint(1024 D) (Secs. II-C, II-D, II-E): for float |x| < 2^22, rint(x) is the
  low mantissa field of the float sum x + 1.5 * 2^23.
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


def _rint_by_add(x):
    """rint of float32 values |x| < 2^22 through one float add of 1.5 * 2^23: the sum's unit in the
    last place is 1, so its low mantissa bits hold rint(x) (ties to even)."""
    s = (np.asarray(x, np.float32) + np.float32(12582912.0)).astype(np.float32)
    return s.view(np.int32).astype(np.int64) - 0x4B400000


def test_rint_by_float_add_matches_rint():
    rng = np.random.default_rng(5)
    lim = 1 << 22
    x = np.concatenate([
        rng.uniform(-lim, lim, 300000),
        rng.normal(0, 300, 100000),                                    # disparity-like values
        np.arange(-2000, 2000) + 0.5,                                  # ties
        np.arange(-2000, 2000) * 1024.0 + 512.0,                       # ties of 1024 x
        [0.0, -0.0, 0.5, -0.5, 1.5, -1.5, 2.5, lim - 0.5, -(lim - 0.5), lim - 1, -(lim - 1)],
    ]).astype(np.float32)
    x = x[np.abs(x) < lim]
    assert np.array_equal(_rint_by_add(x), np.rint(x.astype(np.float64)).astype(np.int64))
    # the scaled inputs of the kernels: rint(1024 * v) for float v, 1024 v exact
    v = rng.normal(0, 40, 200000).astype(np.float32)
    xv = (v * np.float32(1024.0)).astype(np.float32)
    assert np.array_equal(_rint_by_add(xv), np.rint(v.astype(np.float64) * 1024.0).astype(np.int64))
