"""The allocation-free transform entry point, for callers that may not allocate device memory
(code inside a CUDA-graph capture, real-time loops that cannot stall on cudaMalloc / cudaFree,
processes whose device memory belongs to another allocator).  It is called through the C ABI with
no context and must give the results of the ordinary pd_transform, call after call, while the
scratch it reuses (one fixed array inside the library) keeps the previous call's contents.

This file is collected last on purpose, so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process."""
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


def _d1(seed, W, H):
    """A disparity map shaped like the method's D1: a rolled quadratic road with potholes and
    some invalid pixels."""
    sc = synth.road_scaled(W, H, seed)
    D1 = synth.gt_disparity(sc).astype(np.float32)
    rng = np.random.default_rng(seed)
    D1 += rng.normal(0, 0.2, D1.shape).astype(np.float32)
    D1[rng.random(D1.shape) < 0.05] = -1.0
    D1[:, :20] = -1.0
    return D1


def _close_rel(a, b, rel=1e-5, absf=1e-9):
    return abs(a - b) <= rel * max(abs(a), abs(b)) + absf


def _run(B, d1, order, stream=None):
    H, W = d1.shape
    fitted = torch.zeros(64, dtype=torch.uint8, device="cuda")
    D2 = torch.full((H, W), -7.0, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    st = B.pd_transform_noalloc(d1, order, 16.0, fitted, D2, stream=stream)
    assert st == B.PD_OK
    torch.cuda.synchronize()
    assert free_before - torch.cuda.mem_get_info()[0] < (2 << 20)   # no device allocation
    return fitted, D2


@pytest.mark.parametrize("order", [2, 1])
def test_noalloc_transform_matches_the_context_version(orc, B, order):
    """The entry point runs the very kernels of pd_transform on the same data, so the road model
    and D2 are the same bits; the fit also agrees with the oracle (1e-5 relative, D2 1e-4 px).
    Three calls in a row: 640x480, 1280x720 and 2048x2048 (the 4 Mpixel limit)."""
    ctx = B.Context(0)
    for D1 in [_d1(101, 640, 480), _d1(202, 1280, 720), _d1(303, 2048, 2048)]:
        d1 = torch.from_numpy(D1).cuda()
        fitted_ref, D2_ref = B.pd_transform(ctx, d1, order, 16.0)
        fitted, D2 = _run(B, d1, order)
        n = len(bytes(B.RoadModel()))
        assert torch.equal(fitted[:n], fitted_ref[:n])
        assert torch.equal(D2, D2_ref)
        m = B.RoadModel.from_tensor(fitted)
        assert m.order == order
        fit_o = orc.fit_road(orc.moments(D1), order)
        assert _close_rel(m.roll, fit_o.roll, absf=1e-8)
        for i in range(order + 1):
            assert _close_rel(m.a[i], fit_o.a[i])
        D2_o = orc.transform(D1, fit_o, 16.0)
        assert np.max(np.abs(D2.cpu().numpy() - D2_o)) <= 1e-4
    ctx.close()


def test_noalloc_transform_on_a_side_stream(B):
    """Enqueued on a stream other than the current one, the call gives the same bits."""
    ctx = B.Context(0)
    d1 = torch.from_numpy(_d1(404, 960, 540)).cuda()
    fitted_ref, D2_ref = B.pd_transform(ctx, d1, 2, 16.0)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    fitted, D2 = _run(B, d1, 2, stream=side)
    n = len(bytes(B.RoadModel()))
    assert torch.equal(fitted[:n], fitted_ref[:n])
    assert torch.equal(D2, D2_ref)
    ctx.close()


def test_noalloc_transform_rejects_what_does_not_fit(B):
    big = torch.zeros((2049, 2048), dtype=torch.float32, device="cuda")   # > 4 Mpixel
    out = torch.zeros_like(big)
    fitted = torch.zeros(64, dtype=torch.uint8, device="cuda")
    assert B.pd_transform_noalloc(big, 2, 16.0, fitted, out) == B.PD_ERR_INVALID_ARG
    small = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    assert B.pd_transform_noalloc(small, 3, 16.0, fitted, small.clone()) == B.PD_ERR_INVALID_ARG
    torch.cuda.synchronize()
