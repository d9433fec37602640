"""The batched form: many pairs of different sizes and disparity ranges in one call must give
exactly the single-pair results (which the parity tests tie to the oracle), with or without CUDA
graphs, autotuning and multiple scratch waves."""
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


def _items(B, specs, seed0):
    items = []
    for k, (W, H, D) in enumerate(specs):
        sc = synth.road_scaled(W, H, seed0 + k) if (W, H) != (320, 240) else synth.road_320x240(seed0 + k)
        left, right = synth.render(sc)
        items.append((torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda(),
                      B.RoadModel.make(*synth.true_model(sc)), D, sc))
    return items


def _check_against_single(B, ctx, items, outs, paths):
    for (left, right, model, D, _), o in zip(items, outs):
        kap, d_int, D1 = B.pd_sgm(ctx, left, right, model, B.default_params(D=D, paths=paths))
        torch.cuda.synchronize()
        assert torch.equal(o["kappa"], kap)
        assert torch.equal(o["d_int"], d_int)
        assert torch.equal(o["D1"], D1)


SPECS = [(320, 240, 32), (97, 61, 64), (640, 480, 128), (130, 47, 32), (333, 200, 256),
         (1280, 720, 64), (37, 23, 32)]


@pytest.mark.parametrize("paths", [8, 4])
def test_batch_equals_single_pair_calls(B, paths):
    ctx = B.Context(0)
    items = _items(B, SPECS, 300)
    batch = B.make_batch(ctx, [it[:4] for it in items])
    B.pd_sgm_batch(ctx, batch, B.default_params(paths=paths))
    torch.cuda.synchronize()
    _check_against_single(B, ctx, items, batch[1], paths)
    ctx.close()


def test_batch_small_budget_runs_in_waves(B):
    ctx = B.Context(0)
    B.pd_batch_config(ctx, scratch_budget_bytes=64 << 20, use_graph=False, autotune=False)
    items = _items(B, SPECS[:5], 400)
    batch = B.make_batch(ctx, [it[:4] for it in items])
    B.pd_sgm_batch(ctx, batch, B.default_params())
    torch.cuda.synchronize()
    _check_against_single(B, ctx, items, batch[1], 8)
    ctx.close()


def test_batch_graph_replay_with_new_buffers(B):
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = B.Context(0, stream=stream)
        B.pd_batch_config(ctx, use_graph=True, autotune=True)
        for rep in range(3):      # tuning call, capture, replay: same shapes, new data and outputs
            items = _items(B, SPECS[:4], 500 + 10 * rep)
            batch = B.make_batch(ctx, [it[:4] for it in items])
            B.pd_sgm_batch(ctx, batch, B.default_params())
            stream.synchronize()
            _check_against_single(B, ctx, items, batch[1], 8)
            stream.synchronize()
        ctx.close()


def test_batch_matches_oracle_on_a_small_pair(B, orc):
    ctx = B.Context(0)
    items = _items(B, [(97, 61, 32), (320, 240, 32)], 600)
    batch = B.make_batch(ctx, [it[:4] for it in items])
    B.pd_sgm_batch(ctx, batch, B.default_params(paths=8))
    torch.cuda.synchronize()
    for (left, right, model, D, sc), o in zip(items, batch[1]):
        ref = orc.sgm(left.cpu().numpy(), right.cpu().numpy(),
                      orc.RoadModel.make(*synth.true_model(sc)), orc.Params(D=D, paths=8))
        assert np.array_equal(o["d_int"].cpu().numpy(), ref["d_int"])
        assert np.array_equal(o["D1"].cpu().numpy(), ref["D1"])
    ctx.close()


def test_batch_rejects_bad_pairs(B):
    ctx = B.Context(0)
    items = _items(B, [(64, 40, 32)], 700)
    batch = B.make_batch(ctx, [it[:4] for it in items])
    batch[0][0].D = 48
    with pytest.raises(B.PdError) as e:
        B.pd_sgm_batch(ctx, batch, B.default_params())
    assert e.value.status == B.PD_ERR_INVALID_ARG
    ctx.close()


@pytest.mark.slow
def test_benchmark_batch_shapes_in_the_benchmark_configuration(B, orc):
    """The first 16 pairs of the benchmark's mixed batch (resolutions from {640x480, 1280x720,
    1920x1080}, D from {32, 64, 128}, rolls in +-3 deg), run as the benchmark runs them (CUDA
    graph, autotuned block shape, a second replay): every output equals the single-pair call's,
    and a 1920x1080 pair's row shifts, disparities and D1 equal the oracle's."""
    ctx = B.Context(0)
    B.pd_batch_config(ctx, use_graph=True, autotune=True)
    scenes = synth.mixed_batch(16)
    assert {(sc.W, sc.H) for sc, _ in scenes} == {(640, 480), (1280, 720), (1920, 1080)}
    items = []
    for sc, D in scenes:
        left, right = synth.render(sc)
        items.append((torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda(),
                      B.RoadModel.make(*synth.true_model(sc)), D, sc))
    batch = B.make_batch(ctx, [it[:4] for it in items])
    for _ in range(3):          # autotune, capture, replay
        B.pd_sgm_batch(ctx, batch, B.default_params())
    torch.cuda.synchronize()
    _check_against_single(B, ctx, items, batch[1], 8)
    k = next(i for i, (sc, _) in enumerate(scenes) if (sc.W, sc.H) == (1920, 1080))
    sc, D = scenes[k]
    left, right = (t.cpu().numpy() for t in items[k][:2])
    ref = orc.sgm(left, right, orc.RoadModel.make(*synth.true_model(sc)), orc.Params(D=D, paths=8))
    o = batch[1][k]
    assert np.array_equal(o["kappa"].cpu().numpy(), ref["kappa"])
    assert np.array_equal(o["d_int"].cpu().numpy(), ref["d_int"])
    assert np.array_equal(o["D1"].cpu().numpy(), ref["D1"])
    ctx.close()
