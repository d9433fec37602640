"""Closed-loop perspective transformation: each frame's row shifts come from the road model fitted
on the previous frame, on the device (pd_run_pipeline_dev).  The device-model shifts equal the
host-model shifts; over a drive whose roll and offset change every frame, the fits follow the true
road and the residual disparity range after the shift stays narrow."""
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


def test_device_model_gives_the_host_shifts(B, ctx):
    sc = synth.road_scaled(640, 480, 31)
    left, right = (torch.from_numpy(a).cuda() for a in synth.render(sc))
    model = B.RoadModel.make(*synth.true_model(sc))
    p = B.default_params(D=64)
    o1 = B.make_outputs(ctx, 640, 480)
    B.pd_run_pipeline(ctx, left, right, model, p, o1)
    o2 = B.make_outputs(ctx, 640, 480)
    B.pd_run_pipeline_dev(ctx, left, right, B.road_model_tensor(ctx, model), p, o2)
    torch.cuda.synchronize()
    for k in ("kappa", "d_int", "D1", "D2", "labels", "mask"):
        assert torch.equal(o1[1][k], o2[1][k]), k


def test_bad_device_model_gives_zero_shifts(B, ctx):
    sc = synth.road_scaled(320, 240, 32)
    left, right = (torch.from_numpy(a).cuda() for a in synth.render(sc))
    bad = B.RoadModel.make(2, (float("nan"), 0.1, 0.0), 0.0)
    o = B.make_outputs(ctx, 320, 240)
    B.pd_run_pipeline_dev(ctx, left, right, B.road_model_tensor(ctx, bad), B.default_params(D=64), o)
    torch.cuda.synchronize()
    assert (o[1]["kappa"] == 0).all()


def test_closed_loop_follows_the_road(B, ctx):
    W, H, n = 640, 480, 10
    frames = synth.drive_sequence(W, H, n, 40)
    p = B.default_params(D=64)
    outs = B.make_outputs(ctx, W, H)
    model_dev = B.road_model_tensor(ctx, B.RoadModel.make(*synth.true_model(frames[0])))
    for t, sc in enumerate(frames):
        left, right = (torch.from_numpy(a).cuda() for a in synth.render(sc))
        B.pd_run_pipeline_dev(ctx, left, right, model_dev, p, outs)
        torch.cuda.synchronize()
        fit = B.RoadModel.from_tensor(outs[1]["fitted"])
        assert abs(fit.roll - sc.roll) < np.deg2rad(0.1), (t, np.rad2deg(fit.roll - sc.roll))
        d0 = outs[1]["d_int"][outs[1]["D1"] >= 0].float()
        lo, hi = torch.quantile(d0, 0.01).item(), torch.quantile(d0, 0.99).item()
        assert hi - lo < 20, (t, lo, hi)
        model_dev.copy_(outs[1]["fitted"])          # this frame's fit shifts the next frame
