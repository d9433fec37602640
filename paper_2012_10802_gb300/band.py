"""Training and use of the band network (an extension beyond the paper).

The network (cnn.cu) predicts, per 16x16 tile of the row-shifted pair of Sec. II-A, the centre of
the tile's disparities and a confidence; pd_sgm_band then searches [c - 8, c + 8] in confident
tiles and the full range elsewhere.  Training data: synthetic road pairs (the generator of
synth.py, drawn on the GPU), labelled by the full-range SGM of the same library (pd_sgm followed
by pd_band_labels).  Every step of data labelling, the forward and backward passes and the Adam
updates runs in the library's kernels; this module only sequences the calls.

    python -m paper_2012_10802_gb300.band train --pairs 2000 --steps 4000 --out weights.npz
"""
import argparse
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "weights", "band_cnn_1920x1080_d128.npz")
TRAIN_SEED0 = 10000
TEST_SEED0 = 20000


def init_params(seed):
    """He-normal weights (std sqrt(2 / fan_in)), zero biases, in the library's parameter order
    (per layer: weights [Cout][3][3][Cin], then the biases)."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in [(2, 32), (32, 32), (32, 32), (32, 2)]:
        parts.append(rng.normal(0.0, np.sqrt(2.0 / (9 * ci)), size=co * 9 * ci))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


def load_params(path=WEIGHTS):
    with np.load(path) as z:
        return z["params"].astype(np.float32)


def make_training_set(B, ctx, n_pairs, W=1920, H=1080, D=128, seed0=TRAIN_SEED0, log=None):
    """Network inputs [n][Hd][Wd][2] (bf16) and targets [n][th][tw][4] (float) on the device."""
    import torch
    from . import synth

    Hd, Wd, th, tw = (H + 3) // 4, (W + 3) // 4, (H + 15) // 16, (W + 15) // 16
    X = torch.empty((n_pairs, Hd, Wd, 2), dtype=torch.bfloat16, device=ctx.device)
    T = torch.empty((n_pairs, th, tw, 4), dtype=torch.float32, device=ctx.device)
    p = B.default_params(D=D)
    kap = ctx.empty((H,), torch.int32)
    d_int = ctx.empty((H, W), torch.int16)
    D1 = ctx.empty((H, W), torch.float32)
    t0 = time.time()
    for i in range(n_pairs):
        sc = synth.road_scaled(W, H, seed0 + i)
        left, right = synth.render_torch(sc, ctx.device)
        model = B.RoadModel.make(*synth.true_model(sc))
        B.pd_sgm(ctx, left, right, model, p, kap, d_int, D1)
        B.pd_band_input(ctx, left, right, kap, X[i])
        B.pd_band_labels(ctx, d_int, D1, D, T[i])
        if log and (i + 1) % 250 == 0:
            torch.cuda.synchronize()
            log("labelled %d pairs in %.1f s" % (i + 1, time.time() - t0))
    torch.cuda.synchronize()
    return X, T


def train(B, ctx, net, X, T, steps, batch=16, lr=2e-3, seed=0, log=None, first=0, stop=None,
          checkpoint=None, resume=False):
    """Adam over random minibatches; the step size falls by 10x over the last quarter of `steps`.
    Runs steps first .. stop - 1 (stop defaults to `steps`).  checkpoint: a file path; with
    resume=True the network, the Adam state and the minibatch generator are restored from it and
    training continues from its step; at the end the state is saved there.  Training is
    bit-reproducible, so a run split at any step gives the bits of an unbroken one."""
    import torch

    n = X.shape[0]
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    if resume:
        state = B.pd_cnn_load(ctx, net, checkpoint)
        g.set_state(torch.frombuffer(bytearray(state), dtype=torch.uint8))
        first = B.pd_cnn_checkpoint_info(checkpoint)["step"]
    stop = steps if stop is None else stop
    loss = torch.zeros(1, dtype=torch.float32, device=ctx.device)
    xb = torch.empty((batch,) + tuple(X.shape[1:]), dtype=X.dtype, device=ctx.device)
    tb = torch.empty((batch,) + tuple(T.shape[1:]), dtype=T.dtype, device=ctx.device)
    history = []
    t0 = time.time()
    for s in range(first, stop):
        idx = torch.randint(0, n, (batch,), generator=g).to(ctx.device)
        torch.index_select(X, 0, idx, out=xb)
        torch.index_select(T, 0, idx, out=tb)
        step_lr = lr if s < 3 * steps // 4 else lr * 0.1
        B.pd_cnn_train_step(ctx, net, xb, tb, step_lr, loss)
        if (s + 1) % 100 == 0 or s == 0:
            history.append((s + 1, loss.item()))
            if log and (s + 1) % 500 == 0:
                log("step %d loss %.4f (%.1f s)" % (s + 1, history[-1][1], time.time() - t0))
    torch.cuda.synchronize()
    if checkpoint:
        B.pd_cnn_save(ctx, net, checkpoint, g.get_state().numpy().tobytes())
    return history


def disagreement(d_band, D1_band, d_full, D1_full, D):
    """Fraction of pixels with u >= D - 1 (where the full range has a result) whose validity
    differs, or that are valid in both with different integer disparities."""
    import torch

    cols = slice(D - 1, None)
    vb, vf = D1_band[:, cols] >= 0, D1_full[:, cols] >= 0
    diff = (vb != vf) | (vb & vf & (d_band[:, cols] != d_full[:, cols]))
    return diff.float().mean().item()


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    tr = sub.add_parser("train")
    tr.add_argument("--pairs", type=int, default=2000)
    tr.add_argument("--steps", type=int, default=4000)
    tr.add_argument("--batch", type=int, default=16)
    tr.add_argument("--lr", type=float, default=2e-3)
    tr.add_argument("--seed", type=int, default=0)
    tr.add_argument("--out", default=WEIGHTS)
    tr.add_argument("--checkpoint", default=None,
                    help="training checkpoint file, written at the end (and read with --resume)")
    tr.add_argument("--resume", action="store_true",
                    help="continue from --checkpoint: network, Adam state and minibatch generator")
    tr.add_argument("--stop", type=int, default=None,
                    help="stop before this step (then --resume continues the same schedule)")
    a = ap.parse_args(argv)

    import torch
    from . import binding as B

    ctx = B.Context(0)
    log = lambda m: print(m, flush=True)
    X, T = make_training_set(B, ctx, a.pairs, log=log)
    conf = T[..., 1].mean().item()
    log("targets: %.3f of tiles confident, %.3f with a centre" % (conf, T[..., 2].mean().item()))
    net = B.Cnn(0, max_batch=a.batch, max_hd=X.shape[1], max_wd=X.shape[2])
    B.pd_cnn_set_params(ctx, net, init_params(a.seed))
    hist = train(B, ctx, net, X, T, a.steps, a.batch, a.lr, a.seed, log, stop=a.stop,
                 checkpoint=a.checkpoint, resume=a.resume)
    params = B.pd_cnn_get_params(ctx, net)
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    np.savez(a.out, params=params, history=np.array(hist, np.float64),
             pairs=a.pairs, steps=a.steps, batch=a.batch, lr=a.lr, seed=a.seed)
    log("saved %s" % a.out)


if __name__ == "__main__":
    main()
