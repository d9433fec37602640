"""CUDA-graph replay of the whole path (pd_pipeline_config): replayed calls give the same outputs as
directly enqueued ones, a changed call (road model, input buffers, parameters) is captured again,
the closed loop with a device-resident model replays frame after frame, and profiled calls keep
their per-stage times and launch counts."""
import pytest

from paper_2012_10802_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("kappa", "d_int", "D1", "fitted", "D2", "labels", "D3", "thresholds", "mask",
        "components", "comps", "n_comps")


@pytest.fixture(scope="module")
def B():
    from paper_2012_10802_gb300 import binding, build
    build.build()
    return binding


@pytest.fixture(scope="module")
def scene():
    sc = synth.road_scaled(640, 480, 71)
    left, right = (torch.from_numpy(a).cuda() for a in synth.render(sc))
    return sc, left, right


def _run(B, ctx, left, right, model, p, graph, times=1):
    B.pd_pipeline_config(ctx, graph)
    o = B.make_outputs(ctx, 640, 480)
    for _ in range(times):
        B.pd_run_pipeline(ctx, left, right, model, p, o)
    torch.cuda.synchronize()
    return o


def _same(o1, o2):
    """Every output equal; of the component buffer only the records written (n_comps)."""
    for k in KEYS:
        if k == "comps":
            continue
        assert torch.equal(o1[1][k], o2[1][k]), k
    n = int(o1[1]["n_comps"].item())
    rec = o1[1]["comps"].numel() // int(o1[0].max_comps)
    m = max(0, min(n, int(o1[0].max_comps))) * rec
    assert torch.equal(o1[1]["comps"][:m], o2[1]["comps"][:m])


def test_replay_matches_direct_enqueue(B, scene):
    sc, left, right = scene
    ctx = B.Context(0)
    model = B.RoadModel.make(*synth.true_model(sc))
    p = B.default_params(D=64)
    direct = _run(B, ctx, left, right, model, p, False)
    replay = _run(B, ctx, left, right, model, p, True, times=3)
    _same(direct, replay)
    ctx.close()


def test_changed_calls_are_captured_again(B, scene):
    sc, left, right = scene
    ctx = B.Context(0)
    p = B.default_params(D=64)
    model = B.RoadModel.make(*synth.true_model(sc))
    a0, a1, a2 = model.a[0], model.a[1], model.a[2]
    model2 = B.RoadModel.make(2, (a0 + 0.7, a1, a2), model.roll + 0.01)
    o = B.make_outputs(ctx, 640, 480)
    B.pd_pipeline_config(ctx, True)
    B.pd_run_pipeline(ctx, left, right, model, p, o)
    B.pd_run_pipeline(ctx, left, right, model2, p, o)  # new model value: captured again
    torch.cuda.synchronize()
    direct2 = _run(B, ctx, left, right, model2, p, False)
    _same(o, direct2)
    # new input buffers with the same content and new parameters
    l2, r2 = left.clone(), right.clone()
    p2 = B.default_params(D=64, slic_iters=4, fit_iters=1)
    B.pd_pipeline_config(ctx, True)
    B.pd_run_pipeline(ctx, l2, r2, model, p2, o)
    torch.cuda.synchronize()
    direct3 = _run(B, ctx, left, right, model, p2, False)
    _same(o, direct3)
    ctx.close()


def test_closed_loop_replays_with_the_device_model(B, scene):
    sc, left, right = scene
    p = B.default_params(D=64)
    results = []
    for graph in (False, True):
        ctx = B.Context(0)
        B.pd_pipeline_config(ctx, graph)
        o = B.make_outputs(ctx, 640, 480)
        m = B.road_model_tensor(ctx, B.RoadModel.make(*synth.true_model(sc)))
        fits = []
        for _ in range(3):  # the fit of each frame drives the next one's shifts, in place
            B.pd_run_pipeline_dev(ctx, left, right, o[1]["fitted"] if fits else m, p, o)
            fits.append(o[1]["fitted"].clone())
        torch.cuda.synchronize()
        results.append((fits, o))
    (f0, o0), (f1, o1) = results
    for a, b in zip(f0, f1):
        assert torch.equal(a, b)
    _same(o0, o1)


def test_profiled_replays_keep_stage_times(B, scene):
    sc, left, right = scene
    model = B.RoadModel.make(*synth.true_model(sc))
    p = B.default_params(D=64)
    counts = []
    for graph in (False, True):
        ctx = B.Context(0)
        B.pd_pipeline_config(ctx, graph)
        o = B.make_outputs(ctx, 640, 480)
        B.pd_profile_enable(ctx, True)
        for _ in range(3):
            B.pd_run_pipeline(ctx, left, right, model, p, o)
        prof = B.pd_profile_read(ctx)
        B.pd_profile_enable(ctx, False)
        assert prof["calls"] == 3
        for k in ("prep_ms", "aggregate_ms", "disparity_ms", "transform_ms", "superpixel_ms",
                  "mask_ms"):
            assert prof[k] > 0.0, k
        counts.append(prof["launches"])
        ctx.close()
    assert counts[0] == counts[1] > 0
