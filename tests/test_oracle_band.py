"""Pins of the oracle's band-restricted SGM (per-tile disparity windows, an extension of Sec. II-B's
aggregation) against facts that do not depend on the band code: the plain full-range oracle, the
same oracle on a sliced cost volume, closed forms for one-disparity and disjoint windows, and the
bounds Eq. (8) puts on every aggregated value."""
import numpy as np
import pytest

from paper_2012_10802_gb300 import synth


def _cost_volume(orc, W, H, D, seed):
    sc = synth.road_scaled(W, H, seed)
    left, right = synth.render(sc)
    m = orc.RoadModel.make(*synth.true_model(sc))
    kap = orc.kappa(m, W, H, 10.0)
    cst = orc.cost(orc.census(left), orc.census(orc.warp(right, kap)), D)
    return cst, kap


def _tiles(W, H):
    return (H + 15) // 16, (W + 15) // 16


def test_full_range_windows_reproduce_plain_sgm(orc):
    W, H, D = 70, 37, 32
    cst, kap = _cost_volume(orc, W, H, D, 11)
    th, tw = _tiles(W, H)
    lo, hi = orc.band_windows(np.full((th, tw), -1, np.int16), W, H, D)
    assert (lo == 0).all() and (hi == D).all()
    for paths in (4, 8):
        S_ref = orc.aggregate(cst, paths, 4, 32)
        S = orc.aggregate_band(cst, lo, hi, paths, 4, 32)
        assert np.array_equal(S, S_ref)
        d_ref, D1_ref = orc.disparity(S_ref, kap, 1)
        d, D1 = orc.disparity_band(S, lo, hi, kap, 1)
        assert np.array_equal(d, d_ref)
        assert np.array_equal(D1, D1_ref)


@pytest.mark.parametrize("a,b", [(5, 22), (0, 17), (15, 32), (9, 10)])
def test_uniform_window_equals_sgm_on_the_sliced_volume(orc, a, b):
    """With one window [a, b) everywhere, Eq. (8) over the window is Eq. (8) over a volume that
    holds only disparities a..b-1."""
    W, H, D = 53, 29, 32
    cst, kap = _cost_volume(orc, W, H, D, 12)
    lo = np.full((H, W), a, np.int16)
    hi = np.full((H, W), b, np.int16)
    S = orc.aggregate_band(cst, lo, hi, 8, 4, 32)
    S_slice = orc.aggregate(np.ascontiguousarray(cst[:, :, a:b]), 8, 4, 32)
    assert np.array_equal(S[:, :, a:b], S_slice)
    assert (S[:, :, :a] == 0xFFFF).all() and (S[:, :, b:] == 0xFFFF).all()
    d, _ = orc.disparity_band(S, lo, hi, kap, 1)
    assert np.array_equal(d, a + np.argmin(S_slice, axis=2))   # argmin keeps the smallest d


def test_one_disparity_windows_sum_the_costs(orc):
    """A window of one disparity d0 leaves L_r(p, d0) = C(p, d0) on every path (the minimum of
    Eq. (8) is L_r(p - r, d0) itself and is subtracted again), so S = paths * C."""
    W, H, D = 40, 24, 32
    cst, kap = _cost_volume(orc, W, H, D, 13)
    lo = np.full((H, W), 7, np.int16)
    hi = lo + 1
    S = orc.aggregate_band(cst, lo, hi, 8, 4, 32)
    assert np.array_equal(S[:, :, 7], 8 * cst[:, :, 7].astype(np.uint16))
    d, _ = orc.disparity_band(S, lo, hi, kap, 1)
    assert (d == 7).all()


def test_disjoint_window_restarts_with_p2(orc):
    """Where the previous pixel's window shares no disparity with the current one, only the
    m + P2 term of Eq. (8) remains: L_r(p, d) = C(p, d) + P2 on the first column of the tile."""
    W, H, D = 48, 16, 64
    cst, _ = _cost_volume(orc, W, H, D, 14)
    tile_lo = np.array([[0, 40, 3]], np.int16)
    lo, hi = orc.band_windows(tile_lo, W, H, D, 17)
    S = orc.aggregate_band(cst, lo, hi, 1, 4, 32)       # the +u direction alone
    c = cst[:, 16, 40:57].astype(np.uint16)
    assert np.array_equal(S[:, 16, 40:57], c + 32)
    c = cst[:, 32, 3:20].astype(np.uint16)             # [3, 20) against [40, 57): disjoint again
    assert np.array_equal(S[:, 32, 3:20], c + 32)


def test_band_values_obey_eq8_bounds(orc):
    """Every aggregated value lies in [C, C + P2] per path (the minimum of Eq. (8) is at least m
    and at most m + P2), the winner lies in its window, and pixels outside their windows carry
    the 0xFFFF marker."""
    W, H, D = 64, 48, 64
    cst, kap = _cost_volume(orc, W, H, D, 15)
    rng = np.random.default_rng(5)
    th, tw = _tiles(W, H)
    tile_lo = rng.integers(-1, D - 10, size=(th, tw)).astype(np.int16)
    lo, hi = orc.band_windows(tile_lo, W, H, D, 17)
    S = orc.aggregate_band(cst, lo, hi, 8, 4, 32)
    d = np.arange(D)[None, None, :]
    inside = (d >= lo[:, :, None]) & (d < hi[:, :, None])
    c = cst.astype(np.int64)
    assert (S[~inside] == 0xFFFF).all()
    assert (S[inside] >= 8 * c[inside]).all()
    assert (S[inside] <= 8 * (c[inside] + 32)).all()
    d_int, D1 = orc.disparity_band(S, lo, hi, kap, 1)
    assert ((d_int >= lo) & (d_int < hi)).all()
    u = np.arange(W)[None, :]
    assert (D1[u < hi - 1] == -1).all()                 # no full window to the left yet


def test_band_windows_clip_to_the_range(orc):
    tile_lo = np.array([[-1, 0, 120, 200, 5]], np.int16)
    lo, hi = orc.band_windows(tile_lo, 80, 16, 128, 17)
    assert (lo[0, 0], hi[0, 0]) == (0, 128)
    assert (lo[0, 16], hi[0, 16]) == (0, 17)
    assert (lo[0, 32], hi[0, 32]) == (120, 128)
    assert (lo[0, 48], hi[0, 48]) == (127, 128)
    assert (lo[0, 64], hi[0, 64]) == (5, 22)


def test_constant_shift_pair_band_equals_full_range(orc):
    """A pair whose right image is the left one moved by d* pixels: any band that contains d*
    gives the full-range winners and validity wherever the full range has a result (u >= D - 1)."""
    W, H, D, dstar = 160, 48, 64, 11
    rng = np.random.default_rng(8)
    left = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    right = np.roll(left, -dstar, axis=1)              # right(x) = left(x + d*)
    right[:, W - dstar:] = rng.integers(0, 256, size=(H, dstar))
    m = orc.RoadModel.make(1, (10.0, 0.0, 0.0), 0.0)   # kappa = floor(10 - 10) = 0
    p = orc.Params(D=D, paths=8)
    full = orc.sgm(left, right, m, p)
    th, tw = _tiles(W, H)
    rngt = np.random.default_rng(9)
    tile_lo = (dstar - rngt.integers(0, 17, size=(th, tw))).astype(np.int16)
    band = orc.sgm_band(left, right, m, p, np.maximum(tile_lo, 0))
    cols = slice(D - 1, W - 4)                          # away from the right image border
    assert (full["d_int"][2:-2, cols] == dstar).all()
    assert np.array_equal(band["d_int"][:, cols], full["d_int"][:, cols])
    # the aggregated values themselves differ (other windows feed the minima of Eq. (8)), so the
    # sub-pixel step may move D1 inside the winning disparity's +-0.5 interval, but validity agrees
    vb, vf = band["D1"][:, cols] >= 0, full["D1"][:, cols] >= 0
    assert np.array_equal(vb, vf)
    assert np.max(np.abs(band["D1"][:, cols][vf] - full["D1"][:, cols][vf])) <= 1.0
