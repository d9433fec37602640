"""Pins of the oracle's Sec. II-C (road fit, roll, disparity transformation) against the textbook
least-squares plane fit, the closed-form synthetic road, and the exact moment definitions."""
import numpy as np
import pytest

from paper_2012_10802_gb300 import synth


def _moments_bigint(D1):
    """The moment sums by their definition, in Python integers."""
    H, W = D1.shape
    out = {"count": 0, "m": {}, "q": {}, "qq": 0}
    for i in range(5):
        for j in range(5 - i):
            out["m"][(i, j)] = 0
    for i in range(3):
        for j in range(3 - i):
            out["q"][(i, j)] = 0
    for v in range(H):
        for u in range(W):
            d = float(D1[v, u])
            if not d >= 0:
                continue
            q = int(np.rint(d * 1024.0))
            ut, vt = 2 * u - (W - 1), 2 * v - (H - 1)
            out["count"] += 1
            for (i, j) in out["m"]:
                out["m"][(i, j)] += ut ** i * vt ** j
            for (i, j) in out["q"]:
                out["q"][(i, j)] += q * ut ** i * vt ** j
            out["qq"] += q * q
    return out


def test_moments_are_exact(orc):
    rng = np.random.default_rng(0)
    D1 = (rng.random((13, 17)) * 60).astype(np.float32)
    D1[rng.random(D1.shape) < 0.2] = -1.0
    assert orc.moments(D1).export() == _moments_bigint(D1)


def test_moments_exceed_int64(orc):
    """Images a little beyond 1080p need the 128-bit sums for the degree-4 coordinate moments."""
    H, W = 1536, 2048
    D1 = np.full((H, W), 30.0, np.float32)
    e = orc.moments(D1).export()
    assert e["count"] == W * H
    ut = np.arange(W, dtype=object) * 2 - (W - 1)
    assert e["m"][(4, 0)] == H * sum(int(x) ** 4 for x in ut)
    assert e["m"][(4, 0)] > 2 ** 63


def _plane_fit(D1):
    H, W = D1.shape
    v, u = np.mgrid[0:H, 0:W]
    ok = D1 >= 0
    A = np.stack([np.ones(ok.sum()), (v[ok] - (H - 1) / 2.0), (u[ok] - (W - 1) / 2.0)], 1)
    coef, *_ = np.linalg.lstsq(A, D1[ok].astype(np.float64), rcond=None)
    return coef


@pytest.mark.parametrize("roll_deg", [0.0, 1.5, -2.7, 12.0])
def test_linear_fit_is_least_squares_plane(orc, roll_deg):
    """For the linear model, min over (a, phi) of Eq. (4) is the least-squares plane
    d = k0 + kv (v - vc) + ku (u - uc) with kv = a1 cos(phi), ku = -a1 sin(phi)."""
    rng = np.random.default_rng(1)
    H, W = 90, 160
    phi = np.deg2rad(roll_deg)
    v, u = np.mgrid[0:H, 0:W].astype(np.float64)
    vp = (v - (H - 1) / 2) * np.cos(phi) - (u - (W - 1) / 2) * np.sin(phi) + (H - 1) / 2
    D1 = (7.0 + 0.2 * vp + rng.normal(0, 0.3, (H, W))).astype(np.float32)
    D1[rng.random((H, W)) < 0.1] = -1.0
    fit = orc.fit_road(orc.moments(D1), 1)
    k0, kv, ku = _plane_fit(np.round(D1.astype(np.float64) * 1024) / 1024)
    assert abs(fit.roll - np.arctan(-ku / kv)) < 1e-9
    assert abs(fit.a[1] * np.cos(fit.roll) - kv) < 1e-9
    # the roll found is a minimum of E0min (Eq. (12))
    e_star, _ = orc.e0min(orc.moments(D1), 1, fit.roll)
    for dphi in (-1e-3, 1e-3):
        assert orc.e0min(orc.moments(D1), 1, fit.roll + dphi)[0] > e_star


def test_e0min_at_zero_roll_is_v_line_residual(orc):
    """At phi = 0 the linear Eq. (12) is the residual of the v-disparity line fit of Eq. (1)."""
    rng = np.random.default_rng(2)
    H, W = 40, 50
    v = np.mgrid[0:H, 0:W][0].astype(np.float64)
    D1 = (3.0 + 0.1 * v + rng.normal(0, 0.5, (H, W))).astype(np.float32)
    q = np.round(D1.astype(np.float64) * 1024) / 1024
    p = np.polyfit(v.ravel(), q.ravel(), 1)
    resid = np.sum((q.ravel() - np.polyval(p, v.ravel())) ** 2)
    e, _ = orc.e0min(orc.moments(D1), 1, 0.0)
    assert abs(e - resid) < 1e-6 * max(1.0, resid)


@pytest.mark.parametrize("maker", [synth.road_320x240, synth.road_1280x720])
def test_quadratic_fit_recovers_generator_road(orc, maker):
    """Noise-free road disparities of a known quadratic road and roll are fitted back."""
    sc = maker()
    sc.potholes = []
    D1 = synth.gt_disparity(sc).astype(np.float32)
    fit = orc.fit_road(orc.moments(D1), 2)
    assert abs(fit.roll - sc.roll) < 2e-6
    v, u = np.mgrid[0:sc.H, 0:sc.W]
    f = np.array([orc.road_f(fit, sc.W, sc.H, uu, vv) for uu, vv in zip(u.ravel()[::97], v.ravel()[::97])])
    assert np.max(np.abs(f - D1.ravel()[::97])) < 2e-3


def test_e0min_curve_minimum_at_true_roll(orc):
    """The E0min(phi) curve (Fig. 3) has its minimum at the roll the road was generated with."""
    sc = synth.road_320x240()
    D1 = synth.gt_disparity(sc).astype(np.float32)
    mom = orc.moments(D1)
    phis = np.deg2rad(np.linspace(-10, 10, 401))
    e = np.array([orc.e0min(mom, 2, p)[0] for p in phis])
    assert abs(phis[np.argmin(e)] - sc.roll) <= np.deg2rad(0.05) + 1e-12
    assert e[0] > 10 * e.min() and e[-1] > 10 * e.min()


def test_transform_flattens_the_road(orc):
    """Eq. (13): with the fitted road removed, a pothole-free road maps to delta_dt; invalid
    pixels get delta_dt; values are clamped at 0."""
    sc = synth.road_320x240()
    sc.potholes = []
    D1 = synth.gt_disparity(sc).astype(np.float32)
    D1[5, 7] = -1.0
    fit = orc.fit_road(orc.moments(D1), 2)
    D2 = orc.transform(D1, fit, 16.0)
    assert np.max(np.abs(D2 - 16.0)) < 2e-3
    assert D2[5, 7] == 16.0
    D1b = D1.copy()
    D1b[239, 100] = 1.0              # f is about 24.7 px on the bottom row: 1 - 24.7 + 16 < 0
    assert orc.transform(D1b, fit, 16.0)[239, 100] == 0.0
