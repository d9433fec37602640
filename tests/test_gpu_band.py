"""Band-restricted SGM on the GPU against the oracle's band SGM (element by element, bit-exact
d* and D1), and against the full-range pd_sgm where every tile searches the full range."""
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


def _pair(W, H, seed):
    sc = synth.road_scaled(W, H, seed)
    left, right = synth.render(sc)
    return sc, left, right


def _tiles(W, H):
    return (H + 15) // 16, (W + 15) // 16


@pytest.mark.parametrize("W,H,D,paths", [(97, 61, 32, 8), (200, 77, 64, 4), (333, 130, 128, 8),
                                         (300, 40, 256, 8)])
def test_full_range_tiles_equal_pd_sgm(B, ctx, W, H, D, paths):
    sc, left, right = _pair(W, H, 40 + D)
    model = B.RoadModel.make(*synth.true_model(sc))
    p = B.default_params(D=D, paths=paths)
    l, r = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    kap, d_ref, D1_ref = B.pd_sgm(ctx, l, r, model, p)
    tl = torch.full(_tiles(W, H), -1, dtype=torch.int16, device="cuda")
    kap2, d, D1 = B.pd_sgm_band(ctx, l, r, model, p, tl, 17)
    torch.cuda.synchronize()
    assert torch.equal(kap, kap2) and torch.equal(d, d_ref) and torch.equal(D1, D1_ref)


def _random_tiles(W, H, D, seed, frac_full=0.2, centre=None):
    rng = np.random.default_rng(seed)
    th, tw = _tiles(W, H)
    if centre is None:
        lo = rng.integers(0, D, size=(th, tw))
    else:
        lo = np.clip(np.rint(centre + rng.normal(0, 3, size=(th, tw))) - 8, 0, D - 17)
    lo = np.where(rng.random((th, tw)) < frac_full, -1, lo)
    return lo.astype(np.int16)


def _tile_centres(sc, W, H, kap):
    """Ground-truth disparity after the row shift, at each tile centre."""
    th, tw = _tiles(W, H)
    v, u = np.mgrid[0:th, 0:tw] * 16 + 8
    v, u = np.minimum(v, H - 1), np.minimum(u, W - 1)
    return synth.gt_disparity(sc, u.astype(np.float64), v.astype(np.float64)) - kap[v]


@pytest.mark.parametrize("W,H,D,paths,kind", [
    (97, 61, 32, 8, "random"), (200, 77, 64, 4, "random"), (160, 120, 128, 8, "random"),
    (333, 130, 128, 8, "near_truth"), (250, 70, 256, 8, "random"), (64, 48, 64, 8, "all_band")])
def test_band_matches_oracle(B, ctx, orc, W, H, D, paths, kind):
    sc, left, right = _pair(W, H, 60 + W)
    m = synth.true_model(sc)
    kap_o = orc.kappa(orc.RoadModel.make(*m), W, H, 10.0)
    if kind == "near_truth":
        tl = _random_tiles(W, H, D, 7, centre=_tile_centres(sc, W, H, kap_o))
    elif kind == "all_band":
        tl = _random_tiles(W, H, D, 8, frac_full=0.0)
    else:
        tl = _random_tiles(W, H, D, 9)
    ref = orc.sgm_band(left, right, orc.RoadModel.make(*m), orc.Params(D=D, paths=paths), tl, 17)
    p = B.default_params(D=D, paths=paths)
    kap, d, D1 = B.pd_sgm_band(ctx, torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda(),
                               B.RoadModel.make(*m), p, torch.from_numpy(tl).cuda(), 17)
    torch.cuda.synchronize()
    assert np.array_equal(kap.cpu().numpy(), ref["kappa"])
    assert np.array_equal(d.cpu().numpy(), ref["d_int"])
    assert np.array_equal(D1.cpu().numpy(), ref["D1"])


@pytest.mark.parametrize("W,H,D,width,kind", [
    (333, 130, 128, 17, "near_truth"), (250, 70, 256, 17, "random"), (181, 45, 64, 1, "random"),
    (129, 100, 128, 16, "near_truth"), (300, 64, 128, 33, "random")])
def test_all_tiles_banded_match_oracle(B, ctx, orc, W, H, D, width, kind):
    """Every tile banded: the rows then run with one lane per row whenever the windows span at
    most two 16-disparity groups (widths up to 17), across window moves of any size and rows
    past the last warp's end."""
    sc, left, right = _pair(W, H, 70 + W + width)
    m = synth.true_model(sc)
    kap_o = orc.kappa(orc.RoadModel.make(*m), W, H, 10.0)
    centre = _tile_centres(sc, W, H, kap_o) if kind == "near_truth" else None
    tl = _random_tiles(W, H, D, 12 + width, frac_full=0.0, centre=centre)
    ref = orc.sgm_band(left, right, orc.RoadModel.make(*m), orc.Params(D=D, paths=8), tl, width)
    _, d, D1 = B.pd_sgm_band(ctx, torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda(),
                             B.RoadModel.make(*m), B.default_params(D=D), torch.from_numpy(tl).cuda(),
                             width)
    torch.cuda.synchronize()
    assert np.array_equal(d.cpu().numpy(), ref["d_int"])
    assert np.array_equal(D1.cpu().numpy(), ref["D1"])


@pytest.mark.parametrize("width", [1, 5, 16, 33])
def test_band_widths_match_oracle(B, ctx, orc, width):
    W, H, D = 150, 50, 64
    sc, left, right = _pair(W, H, 90 + width)
    m = synth.true_model(sc)
    tl = _random_tiles(W, H, D, 10 + width)
    ref = orc.sgm_band(left, right, orc.RoadModel.make(*m), orc.Params(D=D, paths=8), tl, width)
    _, d, D1 = B.pd_sgm_band(ctx, torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda(),
                             B.RoadModel.make(*m), B.default_params(D=D), torch.from_numpy(tl).cuda(),
                             width)
    torch.cuda.synchronize()
    assert np.array_equal(d.cpu().numpy(), ref["d_int"])
    assert np.array_equal(D1.cpu().numpy(), ref["D1"])


def test_band_1080p_matches_oracle(B, ctx, orc):
    """The benchmark's size (1920x1080, D = 128, 8 paths), windows near the true disparity with a
    fifth of the tiles at full range, compared over the whole frame."""
    W, H, D = 1920, 1080, 128
    sc, left, right = _pair(W, H, 20000)
    m = synth.true_model(sc)
    kap_o = orc.kappa(orc.RoadModel.make(*m), W, H, 10.0)
    tl = _random_tiles(W, H, D, 11, centre=_tile_centres(sc, W, H, kap_o))
    ref = orc.sgm_band(left, right, orc.RoadModel.make(*m), orc.Params(D=D, paths=8), tl, 17)
    _, d, D1 = B.pd_sgm_band(ctx, torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda(),
                             B.RoadModel.make(*m), B.default_params(D=D), torch.from_numpy(tl).cuda(),
                             17)
    torch.cuda.synchronize()
    assert np.array_equal(d.cpu().numpy(), ref["d_int"])
    assert np.array_equal(D1.cpu().numpy(), ref["D1"])


def test_band_rejects_bad_arguments(B, ctx):
    l = torch.zeros((32, 32), dtype=torch.uint8, device="cuda")
    tl = torch.zeros((2, 2), dtype=torch.int16, device="cuda")
    with pytest.raises(B.PdError) as e:
        B.pd_sgm_band(ctx, l, l, B.RoadModel.make(1, (10.0, 0.0, 0.0), 0.0),
                      B.default_params(D=32), tl, 33)
    assert e.value.status == B.PD_ERR_INVALID_ARG
