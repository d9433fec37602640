"""Pins of the band-network oracle (oracle/band_cnn.py) against facts outside it: library
routines (scipy's correlation, torch's bfloat16 conversion and Adam), central finite differences
in float64, closed forms of the Huber and logistic losses, and hand-worked label and window
cases."""
import math

import numpy as np
import pytest

from oracle import band_cnn as bc

scipy_signal = pytest.importorskip("scipy.signal")


def test_parameter_count():
    assert bc.n_params() == (32 * 18 + 32) + 2 * (32 * 288 + 32) + (2 * 288 + 2) == 19682


def test_bf16_round_matches_torch_and_hand_values():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(0, 3, 5000), rng.uniform(-1e4, 1e4, 5000),
                        [0.0, -0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 65504.0]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(bc.bf16_round(x), ref)
    assert bc.bf16_round(np.float32(1.0 + 2 ** -8)) == 1.0                       # tie -> even
    assert bc.bf16_round(np.float32(1.0 + 3 * 2 ** -8)) == np.float32(1.0 + 2 ** -6)  # tie -> even (up)


@pytest.mark.parametrize("stride", [1, 2])
def test_conv3x3_matches_scipy_correlate(stride):
    rng = np.random.default_rng(2)
    B, H, W, ci, co = 2, 11, 14, 3, 4
    x = rng.normal(size=(B, H, W, ci))
    w = rng.normal(size=(co, 3, 3, ci))
    b = rng.normal(size=co)
    y = bc.conv3x3(x, w, b, stride)
    for n in range(B):
        for o in range(co):
            acc = np.full((H, W), b[o])
            for i in range(ci):
                acc = acc + scipy_signal.correlate2d(x[n, :, :, i], w[o, :, :, i], mode="same")
            assert np.allclose(y[n, :, :, o], acc[::stride, ::stride], rtol=1e-12, atol=1e-12)
    assert y.shape[1:3] == ((H - 1) // stride + 1, (W - 1) // stride + 1)


def test_network_shapes_match_the_tile_grid():
    """A 1920x1080 frame: input 270x480, output 68x120 = one cell per 16x16 tile."""
    shape = (270, 480)
    for _, _, s, _ in bc.LAYERS:
        shape = (bc.conv_out(shape[0], s), bc.conv_out(shape[1], s))
    assert shape == ((1080 + 15) // 16, 1920 // 16)


def _problem(seed, B=2, H=20, W=24):
    rng = np.random.default_rng(seed)
    theta = bc.init_params(seed).astype(np.float64)
    theta[-2:] = rng.normal(size=2)           # non-zero output biases
    x = rng.normal(size=(B, H, W, 2))
    Ho, Wo = (H + 3) // 4, (W + 3) // 4
    t = np.zeros((B, Ho, Wo, 4))
    t[..., 0] = rng.uniform(0, 40, size=(B, Ho, Wo))
    t[..., 1] = rng.integers(0, 2, size=(B, Ho, Wo))
    t[..., 2] = rng.integers(0, 2, size=(B, Ho, Wo))
    t[..., 3] = 1.0
    return theta, x, t


def test_gradient_matches_central_differences():
    theta, x, t = _problem(3)
    loss, g = bc.loss_and_grad(theta, x, t)
    rng = np.random.default_rng(4)
    sizes = [co * 9 * ci + co for ci, co, _, _ in bc.LAYERS]
    starts = np.cumsum([0] + sizes)
    idx = []
    for li in range(4):                       # weights and biases of every layer
        idx += list(rng.integers(starts[li], starts[li + 1] - bc.LAYERS[li][1], size=12))
        idx += list(range(starts[li + 1] - bc.LAYERS[li][1], starts[li + 1]))[:3]
    eps = 1e-6
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += eps
        tm[k] -= eps
        fd = (bc.loss_and_grad(tp, x, t)[0] - bc.loss_and_grad(tm, x, t)[0]) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])) + 1e-9, (k, fd, g[k])


def test_loss_closed_forms():
    out = np.zeros((1, 1, 4, 2))
    t = np.zeros((1, 1, 4, 4))
    # centre errors 0.5 and 3 (in units of CENTRE_SCALE px), weights 1; confidence logit 0
    out[0, 0, 0, 0], t[0, 0, 0, 0], t[0, 0, 0, 2] = 0.5, 0.0, 1.0
    out[0, 0, 1, 0], t[0, 0, 1, 0], t[0, 0, 1, 2] = 0.0, 3.0 * bc.CENTRE_SCALE, 1.0
    t[..., 1], t[..., 3] = 1.0, 1.0
    loss, g = bc.loss_and_grad_out(out, t)
    assert abs(loss - ((0.125 + 2.5) / 2 + math.log(2.0))) < 1e-12
    assert abs(g[0, 0, 0, 0] - 0.25) < 1e-12 and abs(g[0, 0, 1, 0] + 0.5) < 1e-12
    assert np.allclose(g[0, 0, :, 1], -0.5 / 4)   # (sigmoid(0) - 1) / 4


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    theta = rng.normal(size=50)
    p = torch.nn.Parameter(torch.tensor(theta, dtype=torch.float64))
    opt = torch.optim.Adam([p], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros(50)
    v = np.zeros(50)
    for step in range(1, 4):
        g = rng.normal(size=50)
        p.grad = torch.tensor(g)
        opt.step()
        theta, m, v = bc.adam_step(theta, m, v, g, step, 1e-2)
    assert np.allclose(theta, p.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_band_input_is_the_block_mean_of_the_shifted_pair():
    rng = np.random.default_rng(6)
    H, W = 16, 24
    left = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    right = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    kap = rng.integers(-3, 6, size=H).astype(np.int32)
    x = bc.band_input(left, right, kap)
    sh = np.stack([right[v, np.clip(np.arange(W) - kap[v], 0, W - 1)] for v in range(H)])
    for c, img in enumerate((left, sh)):
        mean = img.astype(np.float64).reshape(H // 4, 4, W // 4, 4).mean(axis=(1, 3))
        assert np.array_equal(x[:, :, c], bc.bf16_round(((mean - 128.0) / 64.0).astype(np.float32)))
    # a size that is not a multiple of 4 repeats the last row and column
    x2 = bc.band_input(left[:14, :23], right[:14, :23], kap[:14])
    assert x2.shape == (4, 6, 2)
    rows = np.clip(np.arange(12, 16), 0, 13)
    cols = np.clip(np.arange(20, 24), 0, 22)
    s = left[np.ix_(rows, cols)].astype(np.int64).sum()
    assert x2[3, 5, 0] == bc.bf16_round(np.float32((s - 2048) / 1024.0))


def test_labels_hand_cases():
    d = np.zeros((32, 32), np.int16)
    D1 = np.zeros((32, 32), np.float32)
    d[:16, :16] = 20                                   # tile (0,0): all 20 -> centre 20, confident
    d[:16, 16:] = np.arange(256).reshape(16, 16) % 40  # tile (0,1): spread 0..39 -> not confident
    D1[16:, :16] = -1.0                                # tile (1,0): no valid pixels
    D1[16:, 16:] = -1.0
    D1[16:20, 16:32] = 1.0                             # tile (1,1): 64 valid pixels of 0
    lab = bc.labels(d, D1, 2, 2)
    assert tuple(lab[0, 0]) == (20, 1, 1, 1)
    vals = np.sort((np.arange(256) % 40))
    assert lab[0, 1, 0] == vals[127] and tuple(lab[0, 1, 1:]) == (0, 1, 1)
    assert tuple(lab[1, 0]) == (0, 0, 0, 1)
    assert tuple(lab[1, 1]) == (0, 1, 1, 1)
    d[:16, :16][0, :2] = 100                           # 2 of 256 outliers: 99.2 % < 99.5 %
    assert bc.labels(d, D1, 2, 2)[0, 0, 1] == 0
    d[:16, :16][0, 1] = 20                             # 1 of 256: 99.6 %
    assert bc.labels(d, D1, 2, 2)[0, 0, 1] == 1


def test_tile_windows_hand_cases():
    ln9 = np.float32(math.log(9.0))
    out = np.array([[[1.0, ln9], [1.0, np.nextafter(ln9, np.float32(0))],
                     [0.15625, 5.0], [0.1875, 5.0], [-1.0, 5.0], [9.0, 5.0]]], np.float32)
    lo = bc.tile_windows(out, 128)
    # centres 16, -, 2.5 -> 2 (ties to even), 3, -16, 144
    assert lo.tolist() == [[8, -1, 0, 0, 0, 111]]
    out[0, 3, 0] = 1.5625                              # 25 -> 17
    assert bc.tile_windows(out, 128)[0, 3] == 17


def test_tile_windows_left_border_inherits():
    """Unconfident tiles left of column D - 1 take the window of tile column ceil((D-1)/16)."""
    ln9 = np.float32(math.log(9.0))
    out = np.zeros((2, 12, 2), np.float32)
    out[..., 0] = 1.25                                  # centre 20 -> window start 12
    out[..., 1] = ln9
    out[0, :3, 1] = 0.0                                 # unconfident, inside the border (t0 = 2 for D = 32)
    out[1, 2, 1] = 0.0                                  # border tile column itself unconfident
    out[1, 0, 1] = 0.0
    out[0, 5, 1] = 0.0                                  # unconfident outside the border: full range
    lo = bc.tile_windows(out, 32)                       # t0 = 2
    assert lo[0, :3].tolist() == [-1, -1, -1]           # tile t0 unconfident: nothing to inherit
    assert lo[1, :3].tolist() == [-1, 12, -1]
    assert lo[0, 5] == -1                               # outside the border: full range
    out[1, 2, 1] = ln9                                  # tile t0 of row 1 confident again
    assert bc.tile_windows(out, 32)[1, :3].tolist() == [12, 12, 12]
    lo = bc.tile_windows(out, 128)                      # t0 = 8: tiles 0..7 inherit from tile 8
    assert lo[0, :8].tolist() == [12] * 8 and (lo[1] == 12).all()
