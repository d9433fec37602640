"""The Sec. III accuracy report on the GPU against the oracle: exact counts, e_p from exact
counts, e_r within 1e-12 relative (its double-precision sum has no fixed order)."""
import math

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


@pytest.mark.parametrize("H,W,seed", [(37, 53, 1), (720, 1280, 2), (1, 7, 3)])
def test_accuracy_matches_oracle(B, ctx, orc, H, W, seed):
    rng = np.random.default_rng(seed)
    D4 = rng.uniform(2, 60, size=(H, W)).astype(np.float32)
    D4[rng.random((H, W)) < 0.05] = np.nan
    D1 = (D4 + rng.normal(0, 1.5, size=(H, W))).astype(np.float32)
    D1[rng.random((H, W)) < 0.2] = -1.0
    mask = (rng.random((H, W)) < 0.1).astype(np.uint8)
    gt = (rng.random((H, W)) < 0.1).astype(np.uint8) * 3
    ref = orc.accuracy(D1, D4, mask, gt)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    got = B.pd_accuracy(ctx, dev(D1), dev(D4), dev(mask), dev(gt))
    for k in ("q", "tp", "fp", "fn", "tn"):
        assert got[k] == ref[k], k
    for k in ("e_p1", "e_p2", "e_p3", "precision", "recall", "accuracy", "fscore"):
        assert got[k] == ref[k] or (math.isnan(got[k]) and math.isnan(ref[k])), k
    assert math.isclose(got["e_r"], ref["e_r"], rel_tol=1e-12)


def test_empty_cases(B, ctx, orc):
    z = torch.zeros((8, 8), dtype=torch.float32, device="cuda") - 1.0
    m = torch.zeros((8, 8), dtype=torch.uint8, device="cuda")
    got = B.pd_accuracy(ctx, z, z, m, m)
    assert got["q"] == 0 and math.isnan(got["e_r"]) and math.isnan(got["precision"])
    assert got["tn"] == 64 and got["accuracy"] == 1.0
