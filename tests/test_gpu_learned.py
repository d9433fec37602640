"""The trained band network (committed weights) on held-out synthetic 1920x1080 road pairs: the
learned band agrees with the full-range SGM on all but 0.5 % of the pixels that have a full-range
result, searches a narrow window in most tiles, and beats a constant-centre band."""
import numpy as np
import pytest

from paper_2012_10802_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W, H, D = 1920, 1080, 128


@pytest.fixture(scope="module")
def B():
    from paper_2012_10802_gb300 import binding, build
    build.build()
    return binding


@pytest.fixture(scope="module")
def setup(B):
    from paper_2012_10802_gb300 import band
    ctx = B.Context(0)
    net = B.Cnn(0, 1, (H + 3) // 4, (W + 3) // 4)
    B.pd_cnn_set_params(ctx, net, band.load_params())
    yield band, ctx, net
    net.close()
    ctx.close()


@pytest.mark.parametrize("i", range(4))
def test_learned_band_agrees_with_full_range(B, setup, i):
    band, ctx, net = setup
    sc = synth.road_scaled(W, H, band.TEST_SEED0 + i)
    left, right = synth.render_torch(sc, "cuda")
    model = B.RoadModel.make(*synth.true_model(sc))
    p = B.default_params(D=D)
    _, d_full, D1_full = B.pd_sgm(ctx, left, right, model, p)
    tl, _, d, D1 = B.pd_sgm_learned(ctx, net, left, right, model, p, 17)
    torch.cuda.synchronize()
    dis = band.disagreement(d, D1, d_full, D1_full, D)
    banded = (tl >= 0).float().mean().item()
    assert dis <= 0.005, dis
    assert banded >= 0.5, banded
    # a constant-centre band (every tile confident, centred on this frame's own median disparity)
    c0 = int(d_full[D1_full >= 0].float().median().item())
    tl_c = torch.full_like(tl, max(0, min(c0 - 8, D - 17)))
    _, d_c, D1_c = B.pd_sgm_band(ctx, left, right, model, p, tl_c, 17)
    torch.cuda.synchronize()
    assert band.disagreement(d_c, D1_c, d_full, D1_full, D) > dis


def test_learned_band_on_the_numpy_rendered_pair(B, setup):
    """The weights also hold on the CPU-rendered generator (same recipe, other random numbers)."""
    band, ctx, net = setup
    sc = synth.road_1920x1080(3)
    left, right = (torch.from_numpy(a).cuda() for a in synth.render(sc))
    model = B.RoadModel.make(*synth.true_model(sc))
    p = B.default_params(D=D)
    _, d_full, D1_full = B.pd_sgm(ctx, left, right, model, p)
    tl, _, d, D1 = B.pd_sgm_learned(ctx, net, left, right, model, p, 17)
    torch.cuda.synchronize()
    assert band.disagreement(d, D1, d_full, D1_full, D) <= 0.005


def test_learned_path_profiled_and_on_a_user_stream(B, setup):
    """The learned path forks its census onto a second stream of the context and joins it before
    the banded cost: profiled calls and calls on a caller's stream give the same bits as a plain
    call, and count their launches (row shifts, census, network input, four convolutions, windows,
    then the banded cost, aggregation, winner and check)."""
    band, ctx, net = setup
    sc = synth.road_scaled(W, H, band.TEST_SEED0 + 1)
    left, right = synth.render_torch(sc, "cuda")
    model = B.RoadModel.make(*synth.true_model(sc))
    p = B.default_params(D=D)
    ref = [t.clone() for t in B.pd_sgm_learned(ctx, net, left, right, model, p, 17)]
    torch.cuda.synchronize()
    B.pd_profile_enable(ctx, True)
    got = B.pd_sgm_learned(ctx, net, left, right, model, p, 17)
    prof = B.pd_profile_read(ctx)
    B.pd_profile_enable(ctx, False)
    for a, b in zip(ref, got):
        assert torch.equal(a, b)
    assert prof["calls"] == 1 and prof["launches"] == 12
    assert prof["aggregate_ms"] > 0.0 and prof["disparity_ms"] > 0.0
    user = torch.cuda.Stream()
    c2 = B.Context(0, stream=user)
    with torch.cuda.stream(user):
        got2 = B.pd_sgm_learned(c2, net, left, right, model, p, 17)
    user.synchronize()
    for a, b in zip(ref, got2):
        assert torch.equal(a, b)
    c2.close()
