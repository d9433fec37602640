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


@pytest.mark.parametrize("order", [2, 1])
def test_noalloc_transform_matches_the_context_version(B, order):
    ctx = B.Context(0)
    cases = [_d1(101, 640, 480), _d1(202, 1280, 720)]
    for D1 in cases:                       # two calls in a row, different sizes and data
        d1 = torch.from_numpy(D1).cuda()
        fitted_ref, D2_ref = B.pd_transform(ctx, d1, order, 16.0)
        fitted = torch.zeros(fitted_ref.shape, dtype=torch.uint8, device="cuda")
        D2 = torch.full(D2_ref.shape, -7.0, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st = B.pd_transform_noalloc(d1, order, 16.0, fitted, D2)
        assert st == B.PD_OK
        torch.cuda.synchronize()
        assert free_before - torch.cuda.mem_get_info()[0] < (2 << 20)   # no device allocation
        m_ref = B.RoadModel.from_tensor(fitted_ref)
        m = B.RoadModel.from_tensor(fitted)
        assert m.order == order
        assert _close_rel(m.roll, m_ref.roll, absf=1e-8)
        for i in range(order + 1):
            assert _close_rel(m.a[i], m_ref.a[i])
        assert torch.max(torch.abs(D2 - D2_ref)).item() <= 1e-4
    ctx.close()


def test_noalloc_transform_rejects_what_does_not_fit(B):
    big = torch.zeros((2049, 2048), dtype=torch.float32, device="cuda")   # > 4 Mpixel
    out = torch.zeros_like(big)
    fitted = torch.zeros(64, dtype=torch.uint8, device="cuda")
    assert B.pd_transform_noalloc(big, 2, 16.0, fitted, out) == B.PD_ERR_INVALID_ARG
    small = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    assert B.pd_transform_noalloc(small, 3, 16.0, fitted, small.clone()) == B.PD_ERR_INVALID_ARG
    torch.cuda.synchronize()
