"""GPU parity: every stage of the CUDA library, called through the C ABI, against the oracle on the
same seeded inputs.  Integer outputs are compared bit-exact; floating-point ones within the bounds
stated at each test (sub-pixel disparity 1e-3 px, road model and roll 1e-5 relative, SLIC labels
identical on >= 99.9 % of pixels)."""
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
    return B.Context(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t, dtype=None):
    a = t.cpu().numpy()
    return a.view(dtype) if dtype is not None else a


def pair(W, H, seed):
    sc = synth.road_scaled(W, H, seed) if (W, H) not in [(320, 240)] else synth.road_320x240(seed)
    left, right = synth.render(sc)
    return sc, left, right


def omodel(orc, sc):
    return orc.RoadModel.make(*synth.true_model(sc))


def bmodel(B, sc):
    return B.RoadModel.make(*synth.true_model(sc))


SIZES_SGM = [(320, 240, 32, 4), (97, 61, 32, 8), (130, 47, 64, 8), (37, 23, 32, 4),
             (300, 200, 128, 8)]


# ---------------------------------------------------------------------- Sec. II-A

@pytest.mark.parametrize("W,H", [(320, 240), (97, 61), (1, 1), (1280, 720)])
def test_warp_and_kappa_bit_exact(orc, B, ctx, W, H):
    sc, left, right = pair(max(W, 8), max(H, 8), 11)
    right = np.ascontiguousarray(right[:H, :W])
    for order, a, roll in [synth.true_model(sc), (1, (5.0, 0.08, 0.0), -0.3), (2, (40.0, -0.2, 3e-3), 0.25)]:
        om, bm = orc.RoadModel.make(order, a, roll), B.RoadModel.make(order, a, roll)
        kap_o = orc.kappa(om, W, H, 10.0)
        rw, kap = B.pd_warp(ctx, dev(right), bm, 10.0)
        assert np.array_equal(host(kap), kap_o)
        assert np.array_equal(host(rw), orc.warp(right, kap_o))


# ---------------------------------------------------------------------- Sec. II-B cost

@pytest.mark.parametrize("W,H", [(97, 61), (320, 240), (3, 2)])
def test_census_bit_exact(orc, B, ctx, W, H):
    img = np.random.default_rng(W).integers(0, 256, (H, W), dtype=np.uint8)
    assert np.array_equal(host(B.pd_census(ctx, dev(img)), np.uint32), orc.census(img))


@pytest.mark.parametrize("W,H,D", [(97, 61, 32), (320, 240, 37), (64, 40, 128), (5, 3, 1), (300, 20, 256)])
def test_cost_bit_exact(orc, B, ctx, W, H, D):
    rng = np.random.default_rng(D)
    left = rng.integers(0, 256, (H, W), dtype=np.uint8)
    right = rng.integers(0, 256, (H, W), dtype=np.uint8)
    ref = orc.cost(orc.census(left), orc.census(right), D)
    assert np.array_equal(host(B.pd_cost(ctx, dev(left), dev(right), D)), ref)


# ---------------------------------------------------------------------- Eq. (8)

@pytest.mark.parametrize("dx,dy", [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1), (1, -1), (-1, 1)])
@pytest.mark.parametrize("W,H,D", [(97, 61, 32), (45, 71, 64), (33, 9, 128), (19, 5, 256), (1, 1, 32)])
def test_aggregate_dir_bit_exact(orc, B, ctx, dx, dy, W, H, D):
    rng = np.random.default_rng(W * 7 + H + D + dx * 3 + dy)
    cost = rng.integers(0, 25, (H, W, D), dtype=np.uint8)
    ref = orc.aggregate_dir(cost, dx, dy, 4, 32)
    assert np.array_equal(host(B.pd_aggregate_dir(ctx, dev(cost), dx, dy, 4, 32)), ref)


@pytest.mark.parametrize("paths", [4, 8])
@pytest.mark.parametrize("W,H,D,P1,P2", [(97, 61, 32, 4, 32), (64, 48, 64, 10, 120), (40, 30, 128, 1, 2)])
def test_aggregate_bit_exact(orc, B, ctx, paths, W, H, D, P1, P2):
    rng = np.random.default_rng(W + paths + P2)
    cost = rng.integers(0, 25, (H, W, D), dtype=np.uint8)
    ref = orc.aggregate(cost, paths, P1, P2)
    assert np.array_equal(host(B.pd_aggregate(ctx, dev(cost), paths, P1, P2), np.uint16), ref)


# ---------------------------------------------------------------------- Eqs. (9)-(10)

@pytest.mark.parametrize("W,H,D", [(97, 61, 32), (320, 240, 64), (150, 20, 128)])
def test_disparity_bit_exact(orc, B, ctx, W, H, D):
    rng = np.random.default_rng(D + W)
    cost = rng.integers(0, 25, (H, W, D), dtype=np.uint8)
    # a smooth true disparity so the left-right check keeps a mix of valid and invalid pixels
    dtrue = (5 + (np.arange(W)[None, :] // 17 + np.arange(H)[:, None] // 13) % 7)
    for v in range(H):
        for u in range(W):
            cost[v, u, dtrue[v, u]] = rng.integers(0, 3)
    S = orc.aggregate(cost, 8, 4, 32)
    kap = rng.integers(-8, 9, H).astype(np.int32)
    d_ref, D1_ref = orc.disparity(S, kap, 1)
    d_int, D1 = B.pd_disparity(ctx, dev(S.view(np.int16)), dev(kap), 1)
    assert np.array_equal(host(d_int), d_ref)
    assert np.array_equal(host(D1), D1_ref)          # one IEEE division each side: bit-exact
    # Oracle-side sanity, over the columns u >= D - 1 where a pixel can be valid at all (at
    # 150 x 20 with D = 128 that is only 15 % of the image): most pixels there pass the check and
    # find the planted disparity, and no pixel left of that band is valid.
    band = D1_ref[:, D - 1:] >= 0
    assert 0.7 < band.mean() < 1.0
    assert (d_ref[:, D - 1:] == dtrue[:, D - 1:]).mean() > 0.95
    assert not (D1_ref[:, :D - 1] >= 0).any()


@pytest.mark.parametrize("W,H,D,paths", SIZES_SGM)
def test_sgm_fused_bit_exact(orc, B, ctx, W, H, D, paths):
    sc, left, right = pair(W, H, 5)
    p = orc.Params(D=D, paths=paths)
    ref = orc.sgm(left, right, omodel(orc, sc), p)
    params = B.default_params(D=D, paths=paths)
    kap, d_int, D1 = B.pd_sgm(ctx, dev(left), dev(right), bmodel(B, sc), params)
    assert np.array_equal(host(kap), ref["kappa"])
    assert np.array_equal(host(d_int), ref["d_int"])
    assert np.array_equal(host(D1), ref["D1"])


@pytest.mark.parametrize("P1,P2", [(4, 32), (7, 39), (8, 40), (10, 64), (1, 231)])
@pytest.mark.parametrize("D", [64, 128])
def test_sgm_fused_penalty_sweep(orc, B, ctx, P1, P2, D):
    """The fused path over penalties up to the largest P2 whose L still fits a byte (24 + P2 =
    255): every L volume and the disparities stay exact."""
    sc, left, right = pair(200, 96, 13)
    p = orc.Params(D=D, paths=8, P1=P1, P2=P2)
    ref = orc.sgm(left, right, omodel(orc, sc), p)
    params = B.default_params(D=D, paths=8, P1=P1, P2=P2)
    kap, d_int, D1 = B.pd_sgm(ctx, dev(left), dev(right), bmodel(B, sc), params)
    assert np.array_equal(host(d_int), ref["d_int"])
    assert np.array_equal(host(D1), ref["D1"])


@pytest.mark.slow
def test_sgm_fused_bit_exact_720p_d128(orc, B, ctx):
    """The benchmark workload itself: 1280x720, D = 128, 8 paths, in the launch configuration the
    benchmark times."""
    sc = synth.road_1280x720()
    left, right = synth.render(sc)
    ref = orc.sgm(left, right, omodel(orc, sc), orc.Params(D=128, paths=8))
    kap, d_int, D1 = B.pd_sgm(ctx, dev(left), dev(right), bmodel(B, sc), B.default_params())
    assert np.array_equal(host(kap), ref["kappa"])
    assert np.array_equal(host(d_int), ref["d_int"])
    assert np.array_equal(host(D1), ref["D1"])


# ---------------------------------------------------------------------- Sec. II-C

def _sgm_D1(orc, W, H, D, seed):
    sc, left, right = pair(W, H, seed)
    return sc, orc.sgm(left, right, omodel(orc, sc), orc.Params(D=D, paths=8))["D1"]


@pytest.mark.parametrize("W,H", [(320, 240), (97, 61), (1920, 1080)])
def test_moments_bit_exact(orc, B, ctx, W, H):
    rng = np.random.default_rng(W)
    D1 = (rng.random((H, W)) * 120).astype(np.float32)
    D1[rng.random((H, W)) < 0.1] = -1.0
    got = host(B.pd_moments(ctx, dev(D1)))
    ref = orc.moments(D1).export()
    vals = [int(got[2 * i]) % (1 << 64) + (int(got[2 * i + 1]) << 64) for i in range(23)]
    flat = [ref["count"]] + [ref["m"][k] for k in sorted(ref["m"], key=lambda t: (t[0], t[1]))] + \
           [ref["q"][k] for k in sorted(ref["q"], key=lambda t: (t[0], t[1]))] + [ref["qq"]]
    assert vals == flat


def _close_rel(a, b, rel=1e-5, absf=1e-9):
    return abs(a - b) <= rel * max(abs(a), abs(b)) + absf


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("W,H,D", [(320, 240, 32), (640, 480, 64)])
def test_transform_parity(orc, B, ctx, order, W, H, D):
    sc, D1 = _sgm_D1(orc, W, H, D, 21)
    fit_o = orc.fit_road(orc.moments(D1), order)
    D2_o = orc.transform(D1, fit_o, 16.0)
    fitted, D2 = B.pd_transform(ctx, dev(D1), order, 16.0)
    fit = B.RoadModel.from_tensor(fitted)
    assert fit.order == order
    assert _close_rel(fit.roll, fit_o.roll, absf=1e-8)
    for i in range(order + 1):
        assert _close_rel(fit.a[i], fit_o.a[i], absf=1e-9)
    assert np.max(np.abs(host(D2) - D2_o)) <= 1e-4


# ---------------------------------------------------------------------- Sec. II-D/E

def _D2(orc, W, H, D, seed):
    sc, D1 = _sgm_D1(orc, W, H, D, seed)
    fit = orc.fit_road(orc.moments(D1), 2)
    return D1, orc.transform(D1, fit, 16.0)


@pytest.mark.parametrize("W,H,K,iters", [(320, 240, 1000, 10), (97, 61, 40, 3), (320, 240, 60, 0),
                                         (200, 150, 5, 4), (64, 48, 1500, 2)])
def test_superpixels_parity(orc, B, ctx, W, H, K, iters):
    _, D2 = _D2(orc, W, H, 32, 31)
    lab_o, cen_o = orc.slic(D2, K, 10.0, iters)
    D3_o = orc.superpixel_mean(D2, lab_o, cen_o.shape[0])
    labels, D3, centres, n = B.pd_superpixels(ctx, dev(D2), K, 10.0, iters, want_centres=True)
    assert n == cen_o.shape[0]
    lab = host(labels)
    agree = lab == lab_o
    assert agree.mean() >= 0.999
    assert np.array_equal(host(D3)[agree], D3_o[agree])
    if agree.all() and iters > 0:
        assert np.array_equal(host(centres), cen_o)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("W,H", [(320, 240), (97, 61)])
def test_pothole_mask_parity(orc, B, ctx, mode, W, H):
    D1, D2 = _D2(orc, W, H, 32, 41)
    lab, cen = orc.slic(D2, 300, 10.0, 10)
    D3 = orc.superpixel_mean(D2, lab, cen.shape[0])
    rc, t_r, t_s, E2_o = orc.threshold(D2, D1, 2.36, mode)
    E2 = torch.empty(256, dtype=torch.float64, device="cuda")
    mask, thr = B.pd_pothole_mask(ctx, dev(D2), dev(D1), dev(D3), 2.36, mode, E2=E2)
    t = host(thr)
    assert t[0] == t_r and t[1] == t_s
    e = host(E2)
    assert np.array_equal(np.isnan(e), np.isnan(E2_o))
    assert np.array_equal(e[~np.isnan(e)], E2_o[~np.isnan(E2_o)])
    assert np.array_equal(host(mask), orc.mask(D3, t_s))


@pytest.mark.parametrize("W,H", [(3, 3), (2, 40), (40, 2), (31, 17), (32, 10), (61, 66),
                                 (1280, 9)])
def test_pothole_mask_ragged_and_invalid(orc, B, ctx, W, H):
    """Sizes around the histogram's 30-column strips and 8-row chunks (and below the 3x3 window),
    a sloped map with a dip, and 4 % of the pixels without a disparity (D1 < 0)."""
    rng = np.random.default_rng(W * 1000 + H)
    v = np.arange(H, dtype=np.float32)[:, None]
    D2 = (12.0 + 0.05 * v + rng.normal(0.0, 0.3, (H, W))).astype(np.float32)
    D2[H // 3: H // 3 + 3, W // 4: W // 4 + 5] -= 4.0
    D1 = np.where(rng.random((H, W)) < 0.04, -1.0, 1.0).astype(np.float32)
    rc, t_r, t_s, E2_o = orc.threshold(D2, D1, 2.36, 0)
    E2 = torch.empty(256, dtype=torch.float64, device="cuda")
    mask, thr = B.pd_pothole_mask(ctx, dev(D2), dev(D1), dev(D2), 2.36, 0, E2=E2)
    t = host(thr)
    e = host(E2)
    assert np.array_equal(np.isnan(e), np.isnan(E2_o))
    assert np.array_equal(e[~np.isnan(e)], E2_o[~np.isnan(E2_o)])
    if rc == 0:
        assert t[0] == t_r and t[1] == t_s
    else:
        assert np.isnan(t[0]) and t[1] == -np.inf
    assert np.array_equal(host(mask), orc.mask(D2, t[1]))


def test_pothole_mask_threshold_edges(orc, B, ctx):
    """D3 values at and next to t_s in float: the GPU's float comparison against t_s rounded up
    gives the oracle's (double) D3 < t_s for every one of them."""
    D1, D2 = _D2(orc, 320, 240, 32, 41)
    rc, t_r, t_s, _ = orc.threshold(D2, D1, 2.36, 0)
    assert rc == 0
    f = np.float32(t_s)
    vals = [f, np.nextafter(f, np.float32(-np.inf)), np.nextafter(f, np.float32(np.inf)),
            np.float32(t_s - 1e-9), np.float32(t_s + 1e-9), np.float32(-np.inf),
            np.float32(np.inf), np.float32(np.nan), np.float32(0.0)]
    D3 = np.resize(np.array(vals, np.float32), D2.shape).astype(np.float32)
    mask, thr = B.pd_pothole_mask(ctx, dev(D2), dev(D1), dev(D3), 2.36, 0)
    assert host(thr)[1] == t_s
    assert np.array_equal(host(mask), orc.mask(D3, t_s))


def test_pothole_mask_empty_split(orc, B, ctx):
    """A constant map has no threshold with two non-empty clusters: t_r is NaN, no pothole."""
    D2 = np.full((40, 50), 16.0, np.float32)
    D1 = np.ones_like(D2)
    rc, t_r, t_s, _ = orc.threshold(D2, D1, 2.36, 0)
    assert rc == -1
    mask, thr = B.pd_pothole_mask(ctx, dev(D2), dev(D1), dev(D2), 2.36, 0)
    t = host(thr)
    assert np.isnan(t[0]) and t[1] == -np.inf and not host(mask).any()


# ---------------------------------------------------------------------- the whole path

@pytest.mark.parametrize("W,H,D,paths", [(320, 240, 32, 4), (640, 480, 64, 8)])
def test_pipeline_parity(orc, B, ctx, W, H, D, paths):
    sc, left, right = pair(W, H, 51)
    p = orc.Params(D=D, paths=paths, slic_K=1000)
    ref = orc.pipeline(left, right, omodel(orc, sc), p)
    params = B.default_params(D=D, paths=paths)
    outs = B.make_outputs(ctx, W, H)
    times = B.pd_run_pipeline(ctx, dev(left), dev(right), bmodel(B, sc), params, outs, times=True)
    t = outs[1]
    assert np.array_equal(host(t["d_int"]), ref["d_int"])
    assert np.array_equal(host(t["D1"]), ref["D1"])
    fit = B.RoadModel.from_tensor(t["fitted"])
    assert _close_rel(fit.roll, ref["fitted"].roll, absf=1e-8)
    assert np.max(np.abs(host(t["D2"]) - ref["D2"])) <= 1e-4
    lab = host(t["labels"])
    agree = lab == ref["labels"]
    assert agree.mean() >= 0.999
    assert np.array_equal(host(t["mask"])[agree], ref["mask"][agree])
    assert times.total_ms > 0
    # Sec. II-E components of the mask, against the oracle's labelling of its own mask
    recs, n = B.component_records(outs)
    lab_ref, n_ref = orc.ccl(ref["mask"].astype(np.uint8), 8)
    if agree.all() and np.array_equal(host(t["mask"]), ref["mask"]):
        comps_ref = orc.components(lab_ref, ref["labels"], n_ref)
        assert n == n_ref
        got = np.stack([recs[f].astype(np.int64) for f in orc.COMPONENT_FIELDS], axis=1)
        assert np.array_equal(got, comps_ref)
        expect = np.where(lab_ref >= 0, np.searchsorted(comps_ref[:, 0], lab_ref), -1)
        assert np.array_equal(host(t["components"]), expect)
    assert n >= 0   # -1 would mean the union-find hit its iteration limit


# ---------------------------------------------------------------------- errors and edges

def test_invalid_arguments_launch_nothing(B, ctx):
    x = torch.zeros((10, 40), dtype=torch.uint8, device="cuda")
    m = B.RoadModel.make(1, (10.0, 0.0, 0.0), 0.0)
    for over in [dict(D=48), dict(D=0), dict(paths=6), dict(P1=40, P2=32), dict(P2=240)]:
        with pytest.raises(B.PdError) as e:
            B.pd_sgm(ctx, x, x, m, B.default_params(**over))
        assert e.value.status == B.PD_ERR_INVALID_ARG
    bad = B.RoadModel.make(3, (1.0, 0.0, 0.0), 0.0)
    with pytest.raises(B.PdError):
        B.pd_sgm(ctx, x, x, bad, B.default_params(D=32))
    cost = torch.zeros((4, 4, 33), dtype=torch.uint8, device="cuda")
    with pytest.raises(B.PdError):
        B.pd_aggregate_dir(ctx, cost, 1, 0, 4, 32)
    raw = torch.zeros(4 * 4 * 32 + 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.PdError) as e:   # misaligned by one byte: rejected before any launch
        B.pd_aggregate_dir(ctx, raw[1:1 + 512].view(4, 4, 32), 1, 0, 4, 32)
    assert "aligned" in str(e.value)
    torch.cuda.synchronize()
    # the context is still usable
    B.pd_sgm(ctx, x, x, m, B.default_params(D=32))
    torch.cuda.synchronize()


def test_image_narrower_than_disparity_range(orc, B, ctx):
    """W < D: every pixel's search range runs past the left edge, so nothing is valid."""
    sc, left, right = pair(20, 15, 3)
    ref = orc.sgm(left, right, omodel(orc, sc), orc.Params(D=32, paths=8))
    kap, d_int, D1 = B.pd_sgm(ctx, dev(left), dev(right), bmodel(B, sc), B.default_params(D=32))
    assert np.array_equal(host(d_int), ref["d_int"])
    assert np.all(host(D1) == -1.0) and np.all(ref["D1"] == -1.0)
