"""The robust road fit on the GPU (reading R17) against the oracle's: zero iterations is
pd_transform exactly; with refits the fitted road agrees with the oracle's refit to 0.01 px
(the inlier test is taken on each side's own fit, so borderline pixels may differ), and deep
potholes bias it much less than the plain fit."""
import numpy as np
import pytest

from paper_2012_10802_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2012_10802_gb300 import binding, build
    build.build()
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    c = B.Context(0)
    yield c
    c.close()


def _scene_d1(seed, W=640, H=480):
    sc = synth.road_scaled(W, H, seed, n_holes=3)
    for p in sc.potholes:
        p.depth, p.ax, p.ay = 8.0, p.ax * 2.0, p.ay * 2.0
    rng = np.random.default_rng(seed)
    D1 = (synth.gt_disparity(sc) + rng.normal(0, 0.2, (H, W))).astype(np.float32)
    D1[rng.random((H, W)) < 0.1] = -1.0
    return sc, D1


def _max_gap(orc, m1, m2, W, H):
    v, u = np.mgrid[0:H:8, 0:W:8]
    g = [abs(orc.road_f(m1, W, H, a, b) - orc.road_f(m2, W, H, a, b)) for a, b in zip(u.ravel(), v.ravel())]
    return max(g)


def test_zero_iterations_is_the_plain_transform(B, ctx):
    _, D1 = _scene_d1(81)
    d = torch.from_numpy(D1).cuda()
    f0, D20 = B.pd_transform(ctx, d, 2, 16.0)
    f1, D21 = B.pd_transform_robust(ctx, d, 2, 16.0, 0, 1.0)
    torch.cuda.synchronize()
    m0, m1 = B.RoadModel.from_tensor(f0), B.RoadModel.from_tensor(f1)
    assert (m0.order, tuple(m0.a), m0.roll) == (m1.order, tuple(m1.a), m1.roll)
    assert torch.equal(f0, f1)               # padding included: the model is written whole
    assert torch.equal(D20, D21)


@pytest.mark.parametrize("order", [2, 1])
def test_refit_matches_oracle_and_resists_potholes(B, ctx, orc, order):
    sc, D1 = _scene_d1(82)
    d = torch.from_numpy(D1).cuda()
    fr, _ = B.pd_transform_robust(ctx, d, order, 16.0, 2, 1.0)
    fp, _ = B.pd_transform(ctx, d, order, 16.0)
    torch.cuda.synchronize()
    rob = B.RoadModel.from_tensor(fr)
    plain = B.RoadModel.from_tensor(fp)
    ref = orc.fit_robust(D1, order, 2, 1.0)
    to_o = lambda m: orc.RoadModel.make(m.order, tuple(m.a), m.roll)
    assert _max_gap(orc, to_o(rob), ref, 640, 480) < 0.01
    truth = orc.RoadModel.make(*synth.true_model(sc, order))
    if order == 2:
        assert _max_gap(orc, to_o(rob), truth, 640, 480) < 0.5 * _max_gap(orc, to_o(plain), truth, 640, 480)
