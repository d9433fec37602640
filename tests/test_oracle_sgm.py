"""Pins of the oracle's Sec. II-A and II-B steps against facts fixed by the paper or by mathematics:
closed forms, hand-worked examples, brute force on tiny inputs and symmetry invariants."""
import itertools
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Sec. II-A, Eqs. (1), (3), (6)

def test_road_f_matches_printed_eq3_linear(orc):
    """Eq. (3) prints f = a0 + a1 (v cos(phi) - u sin(phi)) (rotation about the origin).  The
    centred form is the same family with a shifted a0; check that identity at many points."""
    W, H = 320, 240
    a0, a1, phi = 5.0, 0.08, np.deg2rad(1.5)
    m = orc.RoadModel.make(1, (a0, a1, 0.0), phi)
    uc, vc = (W - 1) / 2, (H - 1) / 2
    a0_origin = a0 + a1 * (vc - vc * np.cos(phi) + uc * np.sin(phi))
    for u, v in [(0, 0), (319, 0), (0, 239), (319, 239), (160.5, 77.25)]:
        printed = a0_origin + a1 * (v * np.cos(phi) - u * np.sin(phi))
        assert abs(orc.road_f(m, W, H, u, v) - printed) < 1e-12


def test_road_f_zero_roll_is_v_disparity_line(orc):
    """With phi = 0, Eq. (3) reduces to the v-disparity line a0 + a1 v of Eq. (1)."""
    m = orc.RoadModel.make(2, (3.0, 0.1, 2e-4), 0.0)
    for u, v in [(0, 0), (10, 50), (99, 99)]:
        assert abs(orc.road_f(m, 100, 100, u, v) - (3.0 + 0.1 * v + 2e-4 * v * v)) < 1e-12


def _kappa_calculus(order, a, phi, W, H, delta_pt):
    """Minimum of f over x in {0..W-1} located by calculus: f is linear or quadratic in x, so the
    minimum is at an end point or at an integer next to the vertex."""
    uc, vc = (W - 1) / 2, (H - 1) / 2
    out = []
    for v in range(H):
        A = (v - vc) * np.cos(phi) + vc

        def f(x):
            vp = A - (x - uc) * np.sin(phi)
            return a[0] + a[1] * vp + (a[2] * vp * vp if order == 2 else 0.0)

        cands = [0, W - 1]
        if order == 2 and a[2] != 0 and np.sin(phi) != 0:
            vp_star = -a[1] / (2 * a[2])
            x_star = uc + (A - vp_star) / np.sin(phi)
            for x in (np.floor(x_star), np.ceil(x_star)):
                if 0 <= x <= W - 1:
                    cands.append(int(x))
        out.append(min(f(x) for x in cands) - delta_pt)
    return np.array(out)


@pytest.mark.parametrize("order,a,roll_deg", [
    (1, (5.0, 0.08, 0.0), 1.5), (2, (5.0, 0.08, 1e-5), 1.5), (2, (10.0, 0.12, 2e-5), -2.0),
    (2, (50.0, -0.3, 4e-3), 25.0)])
def test_kappa_brute_force_equals_calculus(orc, order, a, roll_deg):
    W, H, dpt = 320, 240, 10.0
    m = orc.RoadModel.make(order, a, np.deg2rad(roll_deg))
    kap = orc.kappa(m, W, H, dpt)
    ref = _kappa_calculus(order, a, np.deg2rad(roll_deg), W, H, dpt)
    near = np.abs(ref - np.round(ref)) < 1e-9
    assert np.array_equal(kap[~near], np.floor(ref[~near]).astype(np.int32))


def test_warp_is_row_shift(orc):
    rng = np.random.default_rng(0)
    H, W = 7, 40
    right = rng.integers(0, 256, (H, W), dtype=np.uint8)
    kap = np.array([-3, 0, 2, 5, 39, -39, 1], np.int32)
    out = orc.warp(right, kap)
    for v in range(H):
        idx = np.clip(np.arange(W) - kap[v], 0, W - 1)
        assert np.array_equal(out[v], right[v][idx])


# ------------------------------------------------------------------- Sec. II-B cost c(p, d)

def test_census_hand_example(orc):
    lines = [l for l in open(os.path.join(GOLDEN, "census_5x5.txt")) if not l.startswith("#")]
    img = np.array([[int(x) for x in lines[i].split()] for i in range(1, 6)], np.uint8)
    code = int(lines[6].split()[1])
    assert int(orc.census(img)[2, 2]) == code


def test_census_constant_and_ramp(orc):
    assert not orc.census(np.full((9, 11), 77, np.uint8)).any()
    ramp = np.tile(np.arange(30, dtype=np.uint8) * 3, (12, 1))
    codes = orc.census(ramp)
    # on a left-to-right ramp exactly the neighbours with dx < 0 are darker
    k, mask = 0, 0
    for dy in range(-2, 3):
        for dx in range(-2, 3):
            if dx == 0 and dy == 0:
                continue
            if dx < 0:
                mask |= 1 << k
            k += 1
    assert np.all(codes[2:-2, 2:-2] == mask)


def test_cost_is_hamming_distance(orc):
    rng = np.random.default_rng(1)
    H, W, D = 5, 23, 16
    cl = rng.integers(0, 1 << 24, (H, W), dtype=np.uint32)
    cr = rng.integers(0, 1 << 24, (H, W), dtype=np.uint32)
    c = orc.cost(cl, cr, D)
    for v in range(H):
        for u in range(W):
            for d in range(D):
                if u - d < 0:
                    assert c[v, u, d] == 24
                else:
                    x = int(cl[v, u]) ^ int(cr[v, u - d])
                    assert c[v, u, d] == bin(x).count("1")


def test_cost_zero_at_true_shift(orc):
    rng = np.random.default_rng(2)
    H, W, dstar = 20, 60, 7
    left = rng.integers(0, 256, (H, W), dtype=np.uint8)
    right = np.empty_like(left)
    right[:, :W - dstar] = left[:, dstar:]
    right[:, W - dstar:] = left[:, -1:]
    c = orc.cost(orc.census(left), orc.census(right), 16)
    inner = c[2:-2, dstar + 2:W - 2, dstar]
    assert not inner.any()


# ------------------------------------------------------------------ Sec. II-B, Eqs. (7)-(8)

def _brute_path(costs, P1, P2):
    """min over all disparity sequences on one path of sum c + P1 [|dd| = 1] + P2 [|dd| > 1],
    the 1-D restriction of the energy E1 of Eq. (7), for each final disparity."""
    n, D = costs.shape
    best = np.full(D, np.iinfo(np.int64).max, np.int64)
    for seq in itertools.product(range(D), repeat=n):
        e = sum(int(costs[i, seq[i]]) for i in range(n))
        for i in range(1, n):
            dd = abs(seq[i] - seq[i - 1])
            e += P1 if dd == 1 else (P2 if dd > 1 else 0)
        best[seq[-1]] = min(best[seq[-1]], e)
    return best


@pytest.mark.parametrize("n,D,P1,P2", [(1, 4, 3, 9), (4, 3, 2, 7), (6, 4, 4, 32), (5, 4, 1, 2)])
def test_aggregation_raw_equals_brute_force(orc, n, D, P1, P2):
    rng = np.random.default_rng(n * 10 + D)
    cst = rng.integers(0, 25, (1, n, D), dtype=np.uint8)
    raw = orc.aggregate_dir_raw(cst, 1, 0, P1, P2)
    for k in range(1, n + 1):
        assert np.array_equal(raw[0, k - 1], _brute_path(cst[0, :k], P1, P2))
    # the same path walked right-to-left, and as a column
    rawr = orc.aggregate_dir_raw(cst, -1, 0, P1, P2)
    assert np.array_equal(rawr[0, 0], _brute_path(cst[0, ::-1], P1, P2))
    col = np.ascontiguousarray(cst.transpose(1, 0, 2))
    assert np.array_equal(orc.aggregate_dir_raw(col, 0, 1, P1, P2)[n - 1, 0], raw[0, n - 1])


@pytest.mark.parametrize("dx,dy", [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1), (1, -1), (-1, 1)])
def test_normalised_aggregation_invariants(orc, dx, dy):
    rng = np.random.default_rng(abs(dx * 3 + dy) + 5)
    cst = rng.integers(0, 25, (9, 13, 8), dtype=np.uint8)
    P1, P2 = 4, 32
    L = orc.aggregate_dir(cst, dx, dy, P1, P2).astype(np.int64)
    raw = orc.aggregate_dir_raw(cst, dx, dy, P1, P2)
    # normalisation shifts every d of a pixel by the same amount
    diff = raw - L
    assert np.all(diff == diff[:, :, :1])
    # bounded by the raw cost plus P2
    assert np.all(L >= cst) and np.all(L <= cst.astype(np.int64) + P2)
    # every pixel whose predecessor is outside starts its path: L = c
    H, W = cst.shape[:2]
    for v in range(H):
        for u in range(W):
            if not (0 <= u - dx < W and 0 <= v - dy < H):
                assert np.array_equal(L[v, u], cst[v, u])


@pytest.mark.parametrize("paths", [4, 8])
def test_aggregate_symmetries(orc, paths):
    """The direction sets are closed under flips and transposition, so S must commute with them."""
    rng = np.random.default_rng(paths)
    cst = rng.integers(0, 25, (11, 17, 8), dtype=np.uint8)
    S = orc.aggregate(cst, paths, 4, 32)
    flip_v = orc.aggregate(cst[::-1].copy(), paths, 4, 32)
    assert np.array_equal(flip_v, S[::-1])
    flip_h = orc.aggregate(cst[:, ::-1].copy(), paths, 4, 32)
    assert np.array_equal(flip_h, S[:, ::-1])
    tr = orc.aggregate(np.ascontiguousarray(cst.transpose(1, 0, 2)), paths, 4, 32)
    assert np.array_equal(tr, S.transpose(1, 0, 2))
    # S is the sum of the per-direction terms
    total = sum(orc.aggregate_dir(cst, dx, dy, 4, 32).astype(np.int64)
                for dx, dy in orc.DIRECTIONS[:paths])
    assert np.array_equal(total, S)


# -------------------------------------------------------------------- Sec. II-B, Eqs. (9)-(10)

def test_disparity_parabola_vertex_and_shift(orc):
    H, W, D = 3, 40, 16
    S = np.full((H, W, D), 500, np.uint16)
    rng = np.random.default_rng(3)
    trip = {}
    for v in range(H):
        for u in range(W):
            d = 5
            a, c = int(rng.integers(1, 40)), int(rng.integers(0, 40))
            S[v, u, d - 1], S[v, u, d], S[v, u, d + 1] = 100 + a, 100, 100 + c
            trip[(v, u)] = [int(S[v, u, d - 1]), 100, int(S[v, u, d + 1])]
    kap = np.array([2, -1, 0], np.int32)
    d_int, D1 = orc.disparity(S, kap, 1)
    assert np.all(d_int == 5)
    for (v, u), (sa, sb, sc) in trip.items():
        # vertex of the parabola through (-1, sa), (0, sb), (1, sc), by a least-squares fit
        p = np.polyfit([-1.0, 0.0, 1.0], [sa, sb, sc], 2)
        vertex = -p[1] / (2 * p[0])
        if u >= D - 1:
            assert abs(D1[v, u] - (5 + vertex + kap[v])) < 1e-5
        else:
            assert D1[v, u] == -1.0


def test_disparity_left_right_check(orc):
    """Right view from the same S: a pixel is kept only when both views agree within lr_tol."""
    H, W, D = 1, 30, 8
    S = np.full((H, W, D), 300, np.uint16)
    dtrue = np.full(W, 3)
    dtrue[15:] = 6                    # a disparity step
    for u in range(W):
        S[0, u, dtrue[u]] = 10
    kap = np.zeros(1, np.int32)
    d_int, D1 = orc.disparity(S, kap, 1)
    assert np.array_equal(d_int[0], dtrue)
    # right pixel x is matched by left u = x + d with S(u, d) small
    dR = np.array([min(range(D), key=lambda d: (S[0, x + d, d] if x + d < W else 1 << 20, d))
                   for x in range(W)])
    expect = np.array([u >= D - 1 and abs(dtrue[u] - dR[u - dtrue[u]]) <= 1
                       for u in range(W)])
    assert np.array_equal(D1[0] >= 0, expect)
    assert np.all(D1[0][expect] == dtrue[expect])


def test_sgm_recovers_planar_shift(orc):
    """A pair related by a constant integer shift gives that disparity almost everywhere."""
    rng = np.random.default_rng(4)
    H, W, dstar = 40, 96, 9
    noise = rng.integers(0, 256, (H + 2, W + 2))
    left = ((sum(noise[dy:dy + H, dx:dx + W] for dy in range(3) for dx in range(3)) + 4) // 9).astype(np.uint8)
    right = np.empty_like(left)
    right[:, :W - dstar] = left[:, dstar:]
    right[:, W - dstar:] = left[:, -1:]
    model = orc.RoadModel.make(1, (10.0, 0.0, 0.0), 0.0)   # kappa = floor(10 - 10) = 0
    p = orc.Params(D=32, paths=8)
    out = orc.sgm(left, right, model, p)
    assert np.all(out["kappa"] == 0)
    inner = out["d_int"][:, dstar + 4:W - 4]
    assert np.mean(inner == dstar) > 0.99
