"""Pins of the oracle's robust road fit (reading R17: Sec. II-C's fit repeated on the inliers of
the previous fit): no iterations is the plain fit; a map with no outliers keeps every pixel and
gives the plain fit exactly; with deep potholes the refit is closer to the true road."""
import numpy as np

from paper_2012_10802_gb300 import synth


def _d1(sc, noise, seed, holes=True):
    D = synth.gt_disparity(sc) if holes else synth.road_disparity(
        sc, *np.mgrid[0:sc.H, 0:sc.W][::-1].astype(np.float64))
    rng = np.random.default_rng(seed)
    return (D + rng.normal(0, noise, D.shape)).astype(np.float32)


def _road_err(orc, m, sc):
    v, u = np.mgrid[0:sc.H, 0:sc.W].astype(np.float64)
    f = np.vectorize(lambda uu, vv: orc.road_f(m, sc.W, sc.H, uu, vv))
    uu, vv = u[::8, ::8], v[::8, ::8]
    return float(np.max(np.abs(f(uu, vv) - synth.road_disparity(sc, uu, vv))))


def test_zero_iterations_is_the_plain_fit(orc):
    sc = synth.road_scaled(320, 240, 71)
    D1 = _d1(sc, 0.3, 1)
    plain = orc.fit_road(orc.moments(D1), 2)
    rob = orc.fit_robust(D1, 2, 0, 2.0)
    assert (rob.roll, tuple(rob.a)) == (plain.roll, tuple(plain.a))


def test_no_outliers_keeps_the_plain_fit(orc):
    sc = synth.road_scaled(320, 240, 72)
    D1 = _d1(sc, 0.2, 2, holes=False)
    plain = orc.fit_road(orc.moments(D1), 2)
    rob = orc.fit_robust(D1, 2, 3, 2.0)                 # 10 sigma: every pixel is an inlier
    assert (rob.roll, tuple(rob.a)) == (plain.roll, tuple(plain.a))


def test_potholes_bias_the_plain_fit_more(orc):
    sc = synth.road_scaled(640, 480, 73, n_holes=3)
    for p in sc.potholes:
        p.depth = 8.0
        p.ax *= 2.0
        p.ay *= 2.0
    D1 = _d1(sc, 0.2, 3)
    plain = orc.fit_road(orc.moments(D1), 2)
    rob = orc.fit_robust(D1, 2, 2, 1.0)
    assert _road_err(orc, rob, sc) < 0.5 * _road_err(orc, plain, sc)
