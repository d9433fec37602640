"""Connected components of the pothole mask on the GPU against the oracle's breadth-first
labelling: identical component numbering (raster order of each component's first pixel),
statistics and fake-pothole flags, on random masks, an oracle pipeline mask, degenerate masks and
a full-HD mask."""
import numpy as np
import pytest

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


def _check(B, ctx, orc, mask, sp, conn, max_comps=1 << 16):
    lab_ref, n_ref = orc.ccl(mask, conn)
    comps_ref = orc.components(lab_ref, sp, n_ref)
    labels, recs, n = B.pd_components(ctx, torch.from_numpy(mask).cuda(),
                                      torch.from_numpy(sp.astype(np.int32)).cuda(), conn, max_comps)
    assert n == n_ref
    roots = comps_ref[:, 0]
    expect = np.where(lab_ref >= 0, np.searchsorted(roots, lab_ref), -1)
    assert np.array_equal(labels.cpu().numpy(), expect)
    k = min(n, max_comps)
    got = np.stack([recs[f].astype(np.int64) for f in orc.COMPONENT_FIELDS], axis=1)
    assert np.array_equal(got, comps_ref[:k])
    return n


@pytest.mark.parametrize("conn", [8, 4])
@pytest.mark.parametrize("H,W,density,seed", [(37, 53, 0.3, 1), (64, 64, 0.55, 2),
                                              (17, 200, 0.45, 3), (240, 320, 0.6, 4),
                                              (1, 97, 0.5, 5), (91, 1, 0.5, 6)])
def test_random_masks_match_oracle(B, ctx, orc, conn, H, W, density, seed):
    rng = np.random.default_rng(seed)
    mask = (rng.random((H, W)) < density).astype(np.uint8)
    sp = (np.arange(H)[:, None] // 7) * 1000 + (np.arange(W)[None, :] // 9)
    _check(B, ctx, orc, mask, sp, conn)


def test_blob_masks_full_hd(B, ctx, orc):
    """Large blobs (long union chains across many blocks) at 1920x1080."""
    rng = np.random.default_rng(7)
    H, W = 1080, 1920
    v, u = np.mgrid[0:H, 0:W]
    mask = np.zeros((H, W), np.uint8)
    for _ in range(40):
        cu, cv = rng.uniform(0, W), rng.uniform(0, H)
        ax, ay = rng.uniform(10, 300), rng.uniform(10, 200)
        mask |= (((u - cu) / ax) ** 2 + ((v - cv) / ay) ** 2 < 1).astype(np.uint8)
    mask |= (rng.random((H, W)) < 0.02).astype(np.uint8)
    sp = (v // 40) * 100 + (u // 40)
    for conn in (8, 4):
        assert _check(B, ctx, orc, mask, sp, conn) > 40


def test_degenerate_masks(B, ctx, orc):
    H, W = 50, 70
    sp = np.zeros((H, W), np.int64)
    assert _check(B, ctx, orc, np.zeros((H, W), np.uint8), sp, 8) == 0
    assert _check(B, ctx, orc, np.ones((H, W), np.uint8), sp, 8) == 1
    checker = ((np.arange(H)[:, None] + np.arange(W)[None, :]) % 2).astype(np.uint8)
    assert _check(B, ctx, orc, checker, sp, 8) == 1
    assert _check(B, ctx, orc, checker, sp, 4) == H * W // 2
    # a serpentine: one component whose union chain visits every row
    snake = np.zeros((H, W), np.uint8)
    snake[::2, :] = 1
    snake[1::4, -1] = 1
    snake[3::4, 0] = 1
    assert _check(B, ctx, orc, snake, sp, 4) == 1


def test_capacity_smaller_than_the_count(B, ctx, orc):
    rng = np.random.default_rng(8)
    mask = (rng.random((64, 64)) < 0.3).astype(np.uint8)
    sp = np.zeros((64, 64), np.int64)
    n = _check(B, ctx, orc, mask, sp, 4, max_comps=10)
    assert n > 10


def test_oracle_pipeline_mask(B, ctx, orc):
    """The mask and superpixels of the oracle's whole path on the 320x240 road."""
    from paper_2012_10802_gb300 import synth
    sc = synth.road_320x240()
    left, right = synth.render(sc)
    res = orc.pipeline(left, right, orc.RoadModel.make(*synth.true_model(sc)),
                       orc.Params(D=32, paths=4))
    mask = res["mask"].astype(np.uint8)
    assert mask.any()
    _check(B, ctx, orc, mask, res["labels"], 8)
