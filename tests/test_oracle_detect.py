"""Pins of the oracle's Sec. II-D (SLIC) and Sec. II-E (threshold, mask) steps, and a sanity run
of the whole oracle path on a synthetic road."""
import json
import os

import numpy as np
import pytest

from paper_2012_10802_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_slic_grid_counts(orc):
    assert orc.slic_grid(1920, 1080, 1000) == (1008, 42, 24)
    assert orc.slic_grid(320, 240, 1000) == (999, 37, 27)
    assert orc.slic_grid(5, 5, 1000) == (25, 5, 5)


def test_slic_first_iteration_on_constant_map_is_voronoi(orc):
    """With a constant D2 the gradient is zero (the seeds stay put) and the distance is purely
    spatial, so one assignment is the nearest-seed (Voronoi) partition, lower index on ties."""
    H, W, K = 61, 97, 40
    D2 = np.full((H, W), 16.0, np.float32)
    labels, _ = orc.slic(D2, K, 10.0, 1)
    n, nx, ny = orc.slic_grid(W, H, K)
    seeds = [(((2 * i + 1) * W) // (2 * nx), ((2 * j + 1) * H) // (2 * ny))
             for j in range(ny) for i in range(nx)]
    sx = np.array([s[0] for s in seeds])
    sy = np.array([s[1] for s in seeds])
    v, u = np.mgrid[0:H, 0:W]
    d2 = (u[..., None] - sx) ** 2 + (v[..., None] - sy) ** 2
    assert np.array_equal(labels, np.argmin(d2, axis=2))


def _bowls(W, H, nx, ny, targets):
    """A D2 map made of one quadratic bowl per grid cell, a (x - x0)^2 + b (y - y0)^2 with the
    bowl's centre (x0, y0) at `targets[k]` for cell k.  The central-difference gradient of Sec.
    II-D is then 16 a^2 (x - x0)^2 + 16 b^2 (y - y0)^2 inside the cell: zero at the bowl's centre
    when that is a pixel, and equal on the two pixels around a half-integer centre.  With
    a = b = 1/4 and half-integer centres every value is exact in float32."""
    D2 = np.zeros((H, W), np.float32)
    v, u = np.mgrid[0:H, 0:W]
    cell = (v * ny // H) * nx + (u * nx // W)
    for k, (x0, y0) in enumerate(targets):
        sel = cell == k
        D2[sel] = (0.25 * (u[sel] - x0) ** 2 + 0.25 * (v[sel] - y0) ** 2 + 4.0).astype(np.float32)
    return D2


def test_slic_seed_moves_to_the_unique_gradient_minimum(orc):
    """Sec. II-D moves each grid seed to the lowest-gradient pixel of its 3x3 neighbourhood.  A
    30x30 map with K = 9 has seeds at (5 + 10 i, 5 + 10 j); each cell holds a bowl whose unique
    gradient minimum is one of the nine offsets of its seed, so with zero iterations the returned
    centres are exactly the moved seeds (and their D2 values).  A seed that moved to the largest
    gradient, a one-sided difference or a swapped offset fails."""
    W = H = 30
    n, nx, ny = orc.slic_grid(W, H, 9)
    assert (n, nx, ny) == (9, 3, 3)
    offs = [(-1, -1), (0, -1), (1, -1), (-1, 0), (0, 0), (1, 0), (-1, 1), (0, 1), (1, 1)]
    seeds = [(5 + 10 * i, 5 + 10 * j) for j in range(3) for i in range(3)]
    targets = [(sx + ox, sy + oy) for (sx, sy), (ox, oy) in zip(seeds, offs)]
    D2 = _bowls(W, H, nx, ny, targets)
    _, centres = orc.slic(D2, 9, 10.0, 0)
    for k, (tx, ty) in enumerate(targets):
        assert (centres[k, 0], centres[k, 1]) == (tx, ty), k
        assert centres[k, 2] == D2[ty, tx]


def test_slic_seed_move_ties(orc):
    """Ties of the seed move: the seed itself wins a tie with any neighbour, even one that comes
    earlier in raster order; between two neighbours the first in raster order (row, then column)
    wins.  Bowl centres on half-integers make the two pixels around them equal minima."""
    W = H = 30
    _, nx, ny = orc.slic_grid(W, H, 9)
    seeds = [(5 + 10 * i, 5 + 10 * j) for j in range(3) for i in range(3)]
    cases = [
        ((-0.5, 0.0), (0, 0)),    # seed ties its left neighbour: the seed stays
        ((0.5, 0.0), (0, 0)),     # seed ties its right neighbour: the seed stays
        ((0.0, -0.5), (0, 0)),    # seed ties the pixel above it: the seed stays
        ((0.5, 1.0), (0, 1)),     # (0, 1) and (1, 1) tie: raster order takes (0, 1)
        ((-0.5, -1.0), (-1, -1)),  # (-1, -1) and (0, -1) tie: (-1, -1) comes first
        ((1.0, -0.5), (1, -1)),   # (1, -1) and (1, 0) tie: the upper row comes first
        ((-1.0, 0.5), (-1, 0)),   # (-1, 0) and (-1, 1) tie
        ((0.0, 0.0), (0, 0)),     # plain minimum at the seed
        ((1.0, 1.0), (1, 1)),     # plain minimum at a corner
    ]
    targets = [(sx + c[0][0], sy + c[0][1]) for (sx, sy), c in zip(seeds, cases)]
    D2 = _bowls(W, H, nx, ny, targets)
    _, centres = orc.slic(D2, 9, 10.0, 0)
    for k, ((sx, sy), (_, (ex, ey))) in enumerate(zip(seeds, cases)):
        assert (centres[k, 0], centres[k, 1]) == (sx + ex, sy + ey), k


def _assign(D2, cx, cy, cv, S, coef, prev):
    """One assignment of Sec. II-D over every centre with the distance in float32, in the
    order dv^2 + (dx^2 + dy^2) coef, the lower index on ties, uncovered pixels unchanged."""
    H, W = D2.shape
    v, u = np.mgrid[0:H, 0:W]
    best = np.full((H, W), np.inf, np.float32)
    lab = prev.copy()
    for k in range(len(cx)):
        fx = (u.astype(np.float32) - cx[k]).astype(np.float32)
        fy = (v.astype(np.float32) - cy[k]).astype(np.float32)
        win = (np.abs(fx) <= S) & (np.abs(fy) <= S)
        dv = (D2 - cv[k]).astype(np.float32)
        dd = dv * dv + (fx * fx + fy * fy) * coef
        take = win & (dd < best)
        best[take] = dd[take]
        lab[take] = k
    return lab


def _means(D2, labels, n, old):
    """Centre update of Sec. II-D in Python integers: the mean of x, y and rint(1024 D2) over
    the members (one double division each, then float32); empty clusters keep their centre."""
    H, W = D2.shape
    q = np.rint(D2.astype(np.float64) * 1024).astype(np.int64)
    out = old.copy()
    for k in range(n):
        ys, xs = np.nonzero(labels == k)
        c = len(xs)
        if c == 0:
            continue
        out[k, 0] = np.float32(int(xs.sum()) / c)
        out[k, 1] = np.float32(int(ys.sum()) / c)
        out[k, 2] = np.float32((int(q[ys, xs].sum()) / c) / 1024.0)
    return out


def test_slic_centre_update_and_second_assignment(orc):
    """The centre update of Sec. II-D, recomputed in Python integers from the oracle's first
    assignment, equals the oracle's centres after one iteration bit for bit; the second
    assignment against those centres gives the oracle's two-iteration labels, whose means are
    its two-iteration centres.  A mean over the wrong coordinate, a dropped 1024 scale or an
    update that skips the pixels' values fails."""
    rng = np.random.default_rng(11)
    H, W, K, m = 48, 64, 12, 10.0
    D2 = (16 + rng.normal(0, 1.5, (H, W))).astype(np.float32)
    D2[20:38, 10:40] -= 6.0
    n, _, _ = orc.slic_grid(W, H, K)
    _, c0 = orc.slic(D2, K, m, 0)
    l1, c1 = orc.slic(D2, K, m, 1)
    assert np.array_equal(_means(D2, l1, n, c0), c1)
    S = np.float32(np.sqrt(W * H / K))
    coef = np.float32(m * m * K / (W * H))
    l2, c2 = orc.slic(D2, K, m, 2)
    assert np.array_equal(_assign(D2, c1[:, 0], c1[:, 1], c1[:, 2], S, coef, l1), l2)
    assert np.array_equal(_means(D2, l2, n, c1), c2)
    assert not np.array_equal(l1, l2)  # the second round changes labels: it is exercised


def test_slic_boundaries_follow_a_deep_step(orc):
    """A pit 20 px deep in a flat map: after the iterations no superpixel straddles its edge."""
    H, W = 120, 160
    D2 = np.full((H, W), 24.0, np.float32)
    D2[40:85, 50:117] = 4.0
    labels, _ = orc.slic(D2, 60, 10.0, 10)
    pit = D2 < 14
    for k in np.unique(labels):
        inside = pit[labels == k]
        assert inside.all() or not inside.any()


def test_superpixel_mean_matches_definition(orc):
    rng = np.random.default_rng(3)
    H, W = 50, 70
    D2 = (rng.random((H, W)) * 30).astype(np.float32)
    labels = rng.integers(0, 12, (H, W)).astype(np.int32)
    D3 = orc.superpixel_mean(D2, labels, 12)
    q = np.rint(D2.astype(np.float64) * 1024)
    for k in range(12):
        assert abs(D3[labels == k][0] - q[labels == k].mean() / 1024) < 1e-6
        assert np.all(D3[labels == k] == D3[labels == k][0])


def _e2_by_definition(D2, D1, k):
    """Eq. (16): sum of squared distances to the two cluster means, with the regions of the
    threshold t = k/8 on the diagonal of the g histogram (g as fixed-point integers)."""
    H, W = D2.shape
    q = np.rint(D2.astype(np.float64) * 1024)
    valid = D1 >= 0
    pts1, pts2 = [], []
    for v in range(1, H - 1):
        for u in range(1, W - 1):
            if not valid[v - 1:v + 2, u - 1:u + 2].all():
                continue
            a = q[v, u]
            b = q[v - 1:v + 2, u - 1:u + 2].sum() - a
            if a < 128 * k and b < 1024 * k:
                pts1.append((a, b))
            elif a >= 128 * k and b >= 1024 * k:
                pts2.append((a, b))
    if not pts1 or not pts2:
        return np.nan, None
    p1, p2 = np.array(pts1), np.array(pts2)
    e = ((p1 - p1.mean(0)) ** 2).sum() + ((p2 - p2.mean(0)) ** 2).sum()
    return e, p2[:, 0].mean() / 1024


def test_threshold_energy_matches_definition(orc):
    rng = np.random.default_rng(4)
    H, W = 40, 60
    D2 = (16 + rng.normal(0, 0.4, (H, W))).astype(np.float32)
    D2[10:25, 20:40] -= 5
    D1 = np.ones((H, W), np.float32)
    D1[0, 0] = D1[30, 30] = -1
    rc, t_r, t_s, E2 = orc.threshold(D2, D1, 2.36, 0)
    assert rc == 0
    for k in [1, 60, 90, 100, 120, 127, 128, 129, 140, 255]:
        e, _ = _e2_by_definition(D2, D1, k)
        if np.isnan(e):
            assert np.isnan(E2[k])
        else:
            assert abs(E2[k] - e) <= 1e-9 * e + 1e-6
    kbest = int(np.nanargmin(E2))
    assert t_r == kbest / 8
    _, road_mean = _e2_by_definition(D2, D1, kbest)
    assert abs(t_s - (road_mean - np.float32(2.36))) < 1e-12


def test_two_level_map_gives_the_pit(orc):
    """Road at 16 px, a plateau pit at 10 px: t_r falls between the levels, t_s is the road level
    minus delta_PD = 2.36 (the value Sec. II-E selects), and the mask is exactly the pit."""
    consts = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    dpd = consts["delta_PD"]["value"]
    H, W = 60, 80
    D2 = np.full((H, W), 16.0, np.float32)
    D2[20:40, 30:55] = 10.0
    D1 = np.ones((H, W), np.float32)
    rc, t_r, t_s, _ = orc.threshold(D2, D1, dpd, 0)
    assert rc == 0 and 10.0 < t_r <= 16.0
    assert abs(t_s - (16.0 - np.float32(dpd))) < 1e-9
    mask = orc.mask(D2, t_s)
    assert np.array_equal(mask.astype(bool), D2 < 12)
    rc, t_r1, t_s1, _ = orc.threshold(D2, D1, dpd, 1)
    assert t_s1 == t_r1 - np.float32(dpd)


@pytest.mark.slow
def test_oracle_pipeline_on_synthetic_road(orc):
    """Sanity (not parity): the oracle path on the 320x240 road recovers its geometry."""
    sc = synth.road_320x240()
    left, right = synth.render(sc)
    order, a, roll = synth.true_model(sc)
    model = orc.RoadModel.make(order, a, roll)
    p = orc.Params(D=32, paths=4)
    out = orc.pipeline(left, right, model, p)
    D1 = out["D1"]
    valid = D1 >= 0
    gt = synth.gt_disparity(sc)
    assert valid.mean() > 0.85
    assert np.median(np.abs(D1[valid] - gt[valid])) < 0.3
    assert abs(out["fitted"].roll - sc.roll) < np.deg2rad(0.15)   # 0.67 px of roll signal at 320 px
    deep = synth.pothole_truth(sc, 2.36)
    assert out["mask"][deep].mean() > 0.5
    assert out["mask"][~synth.pothole_truth(sc, 0.0)].mean() < 0.02
