"""Oracle for the learned disparity band (an extension beyond the paper; TEST INFRASTRUCTURE ONLY).

Plain numpy, float64.  Used only by the tests, the smoke check and the benchmark's CPU-baseline
leg; the CUDA library never calls it and shares no code with it.

What it computes, in this order:

1. The network input: the right image shifted row by row by kappa (the perspective transformation
   of Sec. II-A, Eq. (6)), both images averaged over 4x4 blocks (edge pixels repeated where the
   size is not a multiple of 4), mapped to (sum - 2048) / 1024 and rounded to bfloat16; layout
   [Hd][Wd][2] with channel 0 = left, 1 = shifted right, Hd = ceil(H/4), Wd = ceil(W/4).
2. Four 3x3 convolutions, zero padding 1, strides 1, 2, 2, 1, channels 2 -> 32 -> 32 -> 32 -> 2,
   ReLU after the first three.  The output grid has one cell per 16x16 tile of the full image.
   Output channel 0 is the tile's disparity centre divided by CENTRE_SCALE, channel 1 the logit
   of the confidence that the tile's disparities lie within +-7 of that centre.
3. The loss: Huber (delta 1) on channel 0 against centre / CENTRE_SCALE over the tiles whose
   centre weight is 1, plus the logistic cross-entropy on channel 1 over the tiles whose
   confidence weight is 1, each term averaged over its own tiles.
4. Backward pass of 3 and 2 (plain chain rule) and an Adam step.
5. Labels from a full-range disparity map and the conversion of the network's output into per-tile
   windows for the band SGM.

Parameter vector (float, 19682 values): for each layer, the weights as [Cout][3][3][Cin] followed
by the Cout biases.
"""
import math

import numpy as np

LAYERS = [(2, 32, 1, True), (32, 32, 2, True), (32, 32, 2, True), (32, 2, 1, False)]  # Cin, Cout, stride, ReLU
CENTRE_SCALE = 16.0
BAND = 17                 # [c - 8, c + 8]
CONF_LOGIT = np.float32(math.log(9.0))   # sigmoid(z) >= 0.9  <=>  z >= ln 9
MIN_VALID = 64            # a tile needs this many valid pixels to carry a centre label
LABEL_RADIUS = 7
LABEL_FRACTION = (995, 1000)


def n_params():
    return sum(co * 9 * ci + co for ci, co, _, _ in LAYERS)


def unpack(theta):
    """Splits the flat parameter vector into [(W [Cout][3][3][Cin], b [Cout])] per layer."""
    out, k = [], 0
    for ci, co, _, _ in LAYERS:
        w = theta[k:k + co * 9 * ci].reshape(co, 3, 3, ci)
        k += co * 9 * ci
        b = theta[k:k + co]
        k += co
        out.append((w, b))
    return out


def init_params(seed):
    """He-normal weights (std sqrt(2 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co, _, _ in LAYERS:
        parts.append(rng.normal(0.0, math.sqrt(2.0 / (9 * ci)), size=co * 9 * ci))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


# ----------------------------------------------------------------------------- bfloat16

def bf16_round(x):
    """Rounds to the nearest bfloat16 (ties to even), returned as float32: keep the top 16 bits of
    the float32 pattern after adding half of the dropped part's range, plus one if the kept part
    is odd."""
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


# ----------------------------------------------------------------------------- 1. input

def band_input(left, right, kappa):
    H, W = left.shape
    Hd, Wd = (H + 3) // 4, (W + 3) // 4
    cols = np.arange(W)[None, :] - np.asarray(kappa, np.int64)[:, None]
    shifted = right[np.arange(H)[:, None], np.clip(cols, 0, W - 1)]
    out = np.empty((Hd, Wd, 2), np.float32)
    ys = np.clip(4 * np.arange(Hd)[:, None] + np.arange(4)[None, :], 0, H - 1)   # [Hd][4]
    xs = np.clip(4 * np.arange(Wd)[:, None] + np.arange(4)[None, :], 0, W - 1)   # [Wd][4]
    for c, img in enumerate((left, shifted)):
        img = img.astype(np.int64)
        s = np.zeros((Hd, Wd), np.int64)
        for i in range(4):
            for j in range(4):
                s += img[ys[:, i][:, None], xs[:, j][None, :]]
        out[:, :, c] = (s - 2048).astype(np.float32) / np.float32(1024.0)
    return bf16_round(out)


# ----------------------------------------------------------------------------- 2. network

def conv_out(n, stride):
    return (n - 1) // stride + 1     # 3x3, padding 1


def conv3x3(x, w, b, stride):
    """x [B][H][W][Cin], w [Cout][3][3][Cin] -> [B][Ho][Wo][Cout]:
    y(oy, ox, co) = b(co) + sum over ky, kx, ci of x(s oy + ky - 1, s ox + kx - 1, ci) w(co, ky, kx, ci)."""
    B, H, W, _ = x.shape
    Ho, Wo = conv_out(H, stride), conv_out(W, stride)
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.broadcast_to(b, (B, Ho, Wo, w.shape[0])).astype(np.float64).copy()
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, ky:ky + stride * (Ho - 1) + 1:stride, kx:kx + stride * (Wo - 1) + 1:stride, :]
            y += np.tensordot(patch, w[:, ky, kx, :], axes=([3], [1]))
    return y


def _stored(a, bf16):
    return bf16_round(a.astype(np.float32)).astype(np.float64) if bf16 else a


def forward(theta, x, store_bf16=False):
    """Returns the output [B][Ho][Wo][2] and the per-layer inputs and pre-activations.  With
    store_bf16 the activations between layers are rounded to bfloat16, the storage format of the
    GPU network (its arithmetic is otherwise the same sums)."""
    h = np.asarray(x, np.float64)
    if h.ndim == 3:
        h = h[None]
    cache = []
    for (w, b), (_, _, s, relu) in zip(unpack(np.asarray(theta, np.float64)), LAYERS):
        z = conv3x3(h, w, b, s)
        cache.append((h, z))
        h = _stored(np.maximum(z, 0.0), store_bf16) if relu else z
    return h, cache


# ----------------------------------------------------------------------------- 3. loss

def loss_and_grad_out(out, targets):
    """targets [B][Ho][Wo][4] = (centre in px, confidence label, centre weight, confidence
    weight).  Returns the loss and its gradient with respect to out."""
    out = np.asarray(out, np.float64)
    t = np.asarray(targets, np.float64)
    e = out[..., 0] - t[..., 0] / CENTRE_SCALE
    wc, wb = t[..., 2], t[..., 3]
    nc, nb = max(1.0, wc.sum()), max(1.0, wb.sum())
    a = np.abs(e)
    huber = np.where(a <= 1.0, 0.5 * e * e, a - 0.5)
    z, y = out[..., 1], t[..., 1]
    bce = np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z)))
    loss = float((wc * huber).sum() / nc + (wb * bce).sum() / nb)
    g = np.zeros_like(out)
    g[..., 0] = wc * np.clip(e, -1.0, 1.0) / nc
    g[..., 1] = wb * (1.0 / (1.0 + np.exp(-z)) - y) / nb
    return loss, g


# ----------------------------------------------------------------------------- 4. backward, Adam

def backward(theta, cache, g_out, store_bf16=False):
    """Gradient of the loss with respect to the flat parameter vector.  With store_bf16 the
    gradients with respect to each layer's pre-activation are rounded to bfloat16 (the GPU
    network's storage format)."""
    grads = []
    g = _stored(np.asarray(g_out, np.float64), store_bf16)
    params = unpack(np.asarray(theta, np.float64))
    for li in range(len(LAYERS) - 1, -1, -1):
        _, _, s, _ = LAYERS[li]
        w, _ = params[li]
        h, _ = cache[li]
        dz = g  # already through this layer's ReLU
        B, H, W, _ = h.shape
        Ho, Wo = dz.shape[1:3]
        hp = np.pad(h, ((0, 0), (1, 1), (1, 1), (0, 0)))
        dw = np.zeros_like(w)
        dhp = np.zeros_like(hp)
        for ky in range(3):
            for kx in range(3):
                sl = (slice(None), slice(ky, ky + s * (Ho - 1) + 1, s),
                      slice(kx, kx + s * (Wo - 1) + 1, s), slice(None))
                dw[:, ky, kx, :] = np.tensordot(dz, hp[sl], axes=([0, 1, 2], [0, 1, 2]))
                dhp[sl] += np.tensordot(dz, w[:, ky, kx, :], axes=([3], [0]))
        grads.append((dw, dz.sum(axis=(0, 1, 2))))
        g = dhp[:, 1:H + 1, 1:W + 1, :]
        if li > 0 and LAYERS[li - 1][3]:
            g = _stored(g * (cache[li - 1][1] > 0.0), store_bf16)
    flat = []
    for dw, db in reversed(grads):
        flat += [dw.ravel(), db]
    return np.concatenate(flat)


def loss_and_grad(theta, x, targets, store_bf16=False):
    out, cache = forward(theta, x, store_bf16)
    loss, g = loss_and_grad_out(out, targets)
    return loss, backward(theta, cache, g, store_bf16)


def adam_step(theta, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns the new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


# ----------------------------------------------------------------------------- 5. labels, windows

def labels(d_int, D1, tiles_h, tiles_w):
    """Per 16x16 tile of a full-range result: the lower median c of the valid integer disparities
    (D1 >= 0), the confidence label 1 iff at least MIN_VALID pixels are valid and at least 99.5 %
    of them lie in [c - 7, c + 7], the centre weight 1 iff at least MIN_VALID are valid, and the
    confidence weight 1 everywhere.  Returns [tiles_h][tiles_w][4] float32."""
    H, W = d_int.shape
    out = np.zeros((tiles_h, tiles_w, 4), np.float32)
    for ty in range(tiles_h):
        for tx in range(tiles_w):
            blk_d = d_int[16 * ty:16 * ty + 16, 16 * tx:16 * tx + 16]
            blk_v = D1[16 * ty:16 * ty + 16, 16 * tx:16 * tx + 16] >= 0
            vals = np.sort(blk_d[blk_v].astype(np.int64))
            n = vals.size
            out[ty, tx, 3] = 1.0
            if n < MIN_VALID:
                continue
            c = vals[(n - 1) // 2]
            inside = int(np.count_nonzero(np.abs(vals - c) <= LABEL_RADIUS))
            out[ty, tx, 0] = c
            out[ty, tx, 2] = 1.0
            out[ty, tx, 1] = 1.0 if LABEL_FRACTION[1] * inside >= LABEL_FRACTION[0] * n else 0.0
    return out


def tile_windows(out, D, band=BAND):
    """out [Ho][Wo][2] (float32) -> per-tile window start (int16), -1 for full range: confident
    tiles (logit >= ln 9 in float32) start at rint(CENTRE_SCALE * o0) - 8 (float32 arithmetic,
    ties to even), moved inside [0, D - band].  Unconfident tiles of the left border columns
    tx < t0 = ceil((D - 1) / 16), where the full-range search has no valid pixel and so no label
    exists, take the window of tile (ty, t0) when that tile is confident."""
    o = np.asarray(out, np.float32)
    c = np.rint(o[..., 0] * np.float32(CENTRE_SCALE))
    lo = np.clip(c - (band // 2), 0, max(D - band, 0)).astype(np.int16)
    win = np.where(o[..., 1] >= CONF_LOGIT, lo, np.int16(-1)).astype(np.int16)
    t0 = (D - 1 + 15) // 16
    if t0 < win.shape[1]:
        for tx in range(t0):
            win[:, tx] = np.where(win[:, tx] < 0, win[:, t0], win[:, tx])
    return win
