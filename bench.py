"""Benchmark: stereo pothole-detection path at 1280x720, D = 128, 8 paths on one GB300 per rank.

A step is one pass of the whole path over one synthetic stereo pair: perspective warp, census
cost, 8-path aggregation, winner-take-all / sub-pixel / left-right check, disparity
transformation, SLIC and the adaptive threshold with the pothole mask.  The metric is disparity
throughput W*H*D per second (Mdisp/s) over the whole step.  Inputs are resident in HBM; L2 is
flushed (256 MiB write) before every timed step.  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
HERE = ROOT
sys.path.insert(0, ROOT)

W_, H_, D_, PATHS_ = 1280, 720, 128, 8
WORKLOAD = "road_1280x720_d128_8paths: warp+SGM+transform+SLIC(1000,10,10)+threshold+mask+components"
METRIC = "SGM Mdisp/s (W*H*D/s) at 1280x720 D=128, 8 paths, whole path per step"
# Roofline units of the method (integer SGM is bound by the integer ALUs, not by HBM):
#  - aggregation, Eq. (8): 8 integer operations per (pixel, disparity, path): min of the d-1 and
#    d+1 neighbours, + P1, min with L(d), min with m + P2, + cost, - m, the running minimum m(p)
#    and the accumulation into S;
#  - cost: 2 per (pixel, disparity) (xor, popcount); winner-take-all and right view: 2.
#    So 8R + 4 per (pixel, disparity) for the SGM path, 8R for the aggregation kernel.
#  - bytes: a two-sweep design hands one uint8 partial sum between the sweeps, 2 B per (pixel,
#    disparity), plus about 12 B per pixel of images in and disparities out.
# The integer peak is measured live (pd_int_rate: packed u16x2 DPX instructions, counted in u16
# lanes); the theoretical SMs x 128 lanes x clock is reported beside it.
AGG_OPS_PER_UNIT = 8          # per (pixel, disparity, path)
PATH_EXTRA_OPS = 4            # per (pixel, disparity): cost 2 + winner-take-all 2
PATH_BYTES_PER_PD = 2
PATH_BYTES_PER_PIXEL = 12
SMS = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-pair mixed batch")
    ap.add_argument("--no-band", action="store_true", help="skip the learned-band comparison")
    ap.add_argument("--no-stream", action="store_true", help="skip the closed-loop drive")
    ap.add_argument("--no-graph", action="store_true",
                    help="enqueue every kernel directly instead of replaying the captured path")
    ap.add_argument("--band-size", default=None,
                    help="WxH: only time pd_sgm_band on a road of that size with every tile "
                         "banded around its full-range median (for profiling)")
    ap.add_argument("--size", default=None,
                    help="WxH of a smaller road for profiling captures (not a benchmark line)")
    ap.add_argument("--no-full-hd", action="store_true",
                    help="skip the 1920x1080 whole-path line")
    ap.add_argument("--no-pt-compare", action="store_true",
                    help="skip the with / without perspective-transformation comparison")
    ap.add_argument("--int-peak", action="store_true",
                    help="only measure and print the packed u16x2 integer peak (pd_int_rate)")
    return ap.parse_args()


class Clocks:
    """Samples SM clock and throttle reasons with nvidia-smi while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        cmd = ["nvidia-smi", "-i", str(self.index),
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
               "--format=csv,noheader,nounits", "-lms", "200"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- several ranks (replicas only)
# Frames are independent: each rank processes its own frame with no data-path collective, and
# only the timing is combined.  These helpers are the host logic of that path (tested with gloo
# ranks on the CPU).

def rank_seed(rank):
    """Seed of the synthetic pair of a rank (rank 0 runs the 720p benchmark road, seed 2)."""
    return 2 + rank


def max_over_ranks(value, dist, device):
    """The largest of the ranks' values (the slowest rank bounds the job); value itself without a
    process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mdisp(steps, world, W, H, D, t_ms):
    """Whole-job throughput: the disparities of every rank's frames over the slowest rank's time."""
    return steps * world * W * H * D / (t_ms * 1e-3) / 1e6


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


AGG_SOURCES = ("sgm.cu", "sgm_body.cuh")


def agg_source_sha256():
    h = hashlib.sha256()
    for f in AGG_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2012_10802_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def agg_traffic_record():
    """DRAM bytes per launch of the aggregation kernel from the committed ncu summary, if the
    kernel's sources are unchanged since the counters were taken."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "aggregate_traffic.json")))
        if rec.get("source_sha256") == agg_source_sha256():
            return rec.get("dram_bytes_per_launch_full")
    except (OSError, ValueError):
        pass
    return None


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def oracle_pipeline_time(left, right, model_tuple, rows):
    """Times the oracle's whole path on a band of `rows` rows (single thread)."""
    import oracle
    p = oracle.Params(D=D_, paths=PATHS_, slic_K=max(1, round(1000 * rows / H_)))
    m = oracle.RoadModel.make(*model_tuple)
    t0 = time.perf_counter()
    oracle.pipeline(left[:rows].copy(), right[:rows].copy(), m, p)
    return time.perf_counter() - t0


_REF_FRAME = None


def _ref_init():
    """Worker set-up of the reference arm: the oracle's library and the benchmark frame."""
    global _REF_FRAME
    from paper_2012_10802_gb300 import synth
    import oracle
    oracle.lib()
    sc = synth.road_1280x720()
    left, right = synth.render(sc)
    _REF_FRAME = (left, right, synth.true_model(sc))


def _ref_frame(_):
    """One whole oracle path over the full 1280x720 frame; returns its seconds."""
    left, right, model = _REF_FRAME
    return oracle_pipeline_time(left, right, model, H_)


def run_reference(args, rank, world):
    """The oracle as it stands on the host's cores: each step runs the whole path over the full
    1280x720 benchmark frame once per core, in a process pool started with spawn (independent
    frames, like the ranks of the main line); the value is the disparities of all of a step's
    frames over the step's wall time."""
    if rank != 0:
        return
    import multiprocessing as mp
    cores = cpu_cores()
    with mp.get_context("spawn").Pool(cores, initializer=_ref_init) as pool:
        for _ in range(args.warmup):
            pool.map(_ref_frame, range(cores), chunksize=1)
        t0 = time.perf_counter()
        per = []
        for _ in range(args.steps):
            per += pool.map(_ref_frame, range(cores), chunksize=1)
        total = time.perf_counter() - t0
    val = args.steps * cores * W_ * H_ * D_ / total / 1e6
    sample = ("per step: the full 1280x720 frame (D=128, 8 paths, whole oracle path) once on each "
              "of %d host cores; %.1f s per frame per core" % (cores, statistics.mean(per)))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "Mdisp/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u16+f32",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": val, "unit": "Mdisp/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": "Mdisp/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def bench_batch(B, torch, synth, n_pairs=64, steps=5, seq_steps=2):
    """The mixed batch: n pairs with resolutions from {640x480, 1280x720, 1920x1080} and disparity
    ranges from {32, 64, 128}; one pd_sgm_batch call (CUDA graph, autotuned) against n
    sequential pd_sgm calls, both timed with CUDA events on the library stream, L2 flushed before
    every timed call."""
    scenes = synth.mixed_batch(n_pairs)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(stream):
        ctx = B.Context(torch.cuda.current_device(), stream=stream)
        B.pd_batch_config(ctx, use_graph=True, autotune=True)
        items = []
        for sc, D in scenes:
            left, right = synth.render(sc)
            items.append((torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda(),
                          B.RoadModel.make(*synth.true_model(sc)), D))
        disp = sum(it[0].shape[0] * it[0].shape[1] * it[3] for it in items)
        batch = B.make_batch(ctx, items)
        params = B.default_params()
        for _ in range(3):  # autotune, capture, replay
            B.pd_sgm_batch(ctx, batch, params)
        stream.synchronize()
        ms = []
        for _ in range(steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.pd_sgm_batch(ctx, batch, params)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        outs = [B.pd_sgm(ctx, it[0], it[1], it[2], B.default_params(D=it[3])) for it in items]
        stream.synchronize()
        same = all(torch.equal(o[1], b["d_int"]) and torch.equal(o[2], b["D1"])
                   for o, b in zip(outs, batch[1]))
        seq = []
        for _ in range(seq_steps):
            flush.fill_(2)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for it, o in zip(items, outs):
                B.pd_sgm(ctx, it[0], it[1], it[2], B.default_params(D=it[3]), kappa=o[0],
                         d_int=o[1], D1=o[2])
            e1.record(stream)
            e1.synchronize()
            seq.append(e0.elapsed_time(e1))
        ctx.close()
    tb, ts = statistics.median(ms), statistics.median(seq)
    return {"workload": "%d mixed pairs {640x480,1280x720,1920x1080} x D {32,64,128}, 8 paths" % n_pairs,
            "batched_ms": tb, "batched_frames_per_s": n_pairs / (tb * 1e-3),
            "batched_Mdisp_s": disp / (tb * 1e-3) / 1e6,
            "sequential_ms": ts, "sequential_frames_per_s": n_pairs / (ts * 1e-3),
            "sequential_Mdisp_s": disp / (ts * 1e-3) / 1e6, "speedup": ts / tb,
            "identical_to_sequential": bool(same)}


def bench_stream(B, torch, synth, n=16, graph=True):
    """Closed-loop perspective transformation on a 1280x720 drive of n frames whose roll turns by
    0.1 degree and whose road offset grows every frame: each frame's row shifts come from the
    previous frame's device-resident fit (pd_run_pipeline_dev); the first frame uses the true
    model.  Frames are rendered on the GPU beforehand; the whole sequence is timed with CUDA
    events."""
    W, H = 1280, 720
    frames = synth.drive_sequence(W, H, n, 2)
    pairs = [synth.render_torch(sc, "cuda") for sc in frames]
    ctx = B.Context(torch.cuda.current_device())
    B.pd_pipeline_config(ctx, graph)
    p = B.default_params()
    outs = B.make_outputs(ctx, W, H)
    first = B.road_model_tensor(ctx, B.RoadModel.make(*synth.true_model(frames[0])))
    model_dev = first.clone()
    # each frame is copied into fixed input buffers (as from a camera ring), so the captured path
    # replays frame after frame; the copies are part of the timed frame
    lbuf, rbuf = torch.empty_like(pairs[0][0]), torch.empty_like(pairs[0][1])
    for _ in range(2):   # warm-up of the whole chain
        model_dev.copy_(first)
        for left, right in pairs[:3]:
            lbuf.copy_(left)
            rbuf.copy_(right)
            B.pd_run_pipeline_dev(ctx, lbuf, rbuf, model_dev, p, outs)
    torch.cuda.synchronize()
    model_dev.copy_(first)
    fits, ranges = [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total = 0.0
    for (left, right) in pairs:
        e0.record()
        lbuf.copy_(left)
        rbuf.copy_(right)
        B.pd_run_pipeline_dev(ctx, lbuf, rbuf, model_dev, p, outs)
        model_dev.copy_(outs[1]["fitted"])
        e1.record()
        e1.synchronize()
        total += e0.elapsed_time(e1)
        fits.append(B.RoadModel.from_tensor(outs[1]["fitted"]))
        d0 = outs[1]["d_int"][outs[1]["D1"] >= 0].float()
        ranges.append(torch.quantile(d0, 0.99).item() - torch.quantile(d0, 0.01).item())
    ctx.close()
    import math
    roll_err = [abs(math.degrees(f.roll - sc.roll)) for f, sc in zip(fits, frames)]
    return {"workload": "closed-loop drive 1280x720 D=128 8 paths, %d frames, roll +0.1 deg and "
                        "a0 +0.05 px per frame" % n,
            "ms_per_frame": total / n, "max_roll_error_deg": max(roll_err),
            "residual_range_px_p1_p99_max": max(ranges)}


def band_only(B, torch, synth, size, steps, warmup):
    """pd_sgm_band at W x H, D = 128, 8 paths, every tile banded with a 17-disparity window around
    its full-range median (the learned band's common case); prints one JSON line."""
    W, H = (int(x) for x in size.lower().split("x"))
    D = 128
    ctx = B.Context(torch.cuda.current_device())
    sc = synth.road_scaled(W, H, 20000)
    left, right = synth.render_torch(sc, "cuda")
    model = B.RoadModel.make(*synth.true_model(sc))
    p = B.default_params(D=D)
    kap, d_full, D1_full = B.pd_sgm(ctx, left, right, model, p)
    th, tw = (H + 15) // 16, (W + 15) // 16
    pad = torch.nn.functional.pad(d_full.float(), (0, tw * 16 - W, 0, th * 16 - H), value=float("nan"))
    med = torch.nanmedian(pad.reshape(th, 16, tw, 16).permute(0, 2, 1, 3).reshape(th, tw, 256), 2)
    tile_lo = torch.clamp(torch.round(med.values) - 8, 0, D - 17).to(torch.int16)
    d_int, D1 = torch.empty_like(d_full), torch.empty_like(D1_full)
    for _ in range(warmup):
        B.pd_sgm_band(ctx, left, right, model, p, tile_lo, 17, kap, d_int, D1)
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        B.pd_sgm_band(ctx, left, right, model, p, tile_lo, 17, kap, d_int, D1)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    ctx.close()
    print(json.dumps({"workload": "pd_sgm_band %dx%d D=128 8 paths, every tile banded" % (W, H),
                      "ms_median": statistics.median(ms), "steps": steps}))


def bench_band(B, torch, synth, steps=10, n_eval=4):
    """The learned band at 1920x1080, D = 128, 8 paths: the band network (committed weights,
    trained on 2000 synthetic pairs by the library's own kernels) picks a 17-disparity window per
    16x16 tile, against the full-range SGM on the same pairs.  Times are CUDA-event medians on the
    library stream with L2 flushed before each call; disagreement is the fraction of pixels with
    u >= D - 1 whose validity or (valid) integer disparity differs from the full range."""
    from paper_2012_10802_gb300 import band
    W, H, D = 1920, 1080, 128
    if not os.path.exists(band.WEIGHTS):
        return {"unavailable": "no trained weights at " + os.path.relpath(band.WEIGHTS, HERE)}
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(stream):
        ctx = B.Context(torch.cuda.current_device(), stream=stream)
        net = B.Cnn(torch.cuda.current_device(), 1, (H + 3) // 4, (W + 3) // 4)
        B.pd_cnn_set_params(ctx, net, band.load_params())
        p = B.default_params(D=D)
        dis, frac, const_dis, pairs = [], [], [], []
        for i in range(n_eval):
            sc = synth.road_scaled(W, H, band.TEST_SEED0 + i)
            left, right = synth.render_torch(sc, "cuda")
            model = B.RoadModel.make(*synth.true_model(sc))
            pairs.append((left, right, model))
            kap, d_full, D1_full = B.pd_sgm(ctx, left, right, model, p)
            tl, _, d, D1 = B.pd_sgm_learned(ctx, net, left, right, model, p, 17)
            dis.append(band.disagreement(d, D1, d_full, D1_full, D))
            frac.append((tl >= 0).float().mean().item())
            c0 = int(d_full[D1_full >= 0].float().median().item())
            tl_c = torch.full_like(tl, max(0, min(c0 - 8, D - 17)))
            _, d_c, D1_c = B.pd_sgm_band(ctx, left, right, model, p, tl_c, 17)
            const_dis.append(band.disagreement(d_c, D1_c, d_full, D1_full, D))

        def timed(fn):
            for _ in range(3):
                fn()
            ms = []
            for _ in range(steps):
                flush.fill_(3)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            return statistics.median(ms)

        left, right, model = pairs[0]
        kap, d_int, D1 = B.pd_sgm(ctx, left, right, model, p)
        tl = ctx.empty(((H + 15) // 16, (W + 15) // 16), torch.int16)
        x = B.pd_band_input(ctx, left, right, kap)
        out = B.pd_cnn_forward(ctx, net, x)
        full_ms = timed(lambda: B.pd_sgm(ctx, left, right, model, p, kap, d_int, D1))
        learned_ms = timed(lambda: B.pd_sgm_learned(ctx, net, left, right, model, p, 17, tl, kap,
                                                    d_int, D1))
        cnn_ms = timed(lambda: (B.pd_band_input(ctx, left, right, kap, x),
                                B.pd_cnn_forward(ctx, net, x, out)))
        band_only_ms = timed(lambda: B.pd_sgm_band(ctx, left, right, model, p, tl, 17, kap, d_int,
                                                   D1))
        net.close()
        # one Adam step of the network at its training configuration (16 pairs' inputs per step)
        Hd, Wd, Bt = (H + 3) // 4, (W + 3) // 4, 16
        tnet = B.Cnn(torch.cuda.current_device(), Bt, Hd, Wd)
        B.pd_cnn_set_params(ctx, tnet, band.load_params())
        gen = torch.Generator(device="cuda").manual_seed(7)
        xt = torch.randn((Bt, Hd, Wd, 2), generator=gen, device="cuda").to(torch.bfloat16)
        Ho, Wo = (Hd + 3) // 4, (Wd + 3) // 4
        tt = torch.zeros((Bt, Ho, Wo, 4), dtype=torch.float32, device="cuda")
        tt[..., 0] = torch.randint(0, D, (Bt, Ho, Wo), generator=gen, device="cuda").float()
        tt[..., 2:] = 1.0
        lt = torch.zeros(1, dtype=torch.float32, device="cuda")
        train_ms = timed(lambda: B.pd_cnn_train_step(ctx, tnet, xt, tt, 1e-4, lt))
        B.pd_cnn_check(ctx, tnet)
        tnet.close()
        ctx.close()
    disp = W * H * D
    return {"workload": "road_1920x1080_d128_8paths, learned 17-disparity band per 16x16 tile "
                        "(conf >= 0.9) vs full range; %d test pairs" % n_eval,
            "full_range_ms": full_ms, "learned_ms": learned_ms, "speedup": full_ms / learned_ms,
            "learned_Mdisp_s": disp / (learned_ms * 1e-3) / 1e6,
            "full_range_Mdisp_s": disp / (full_ms * 1e-3) / 1e6,
            "cnn_ms": cnn_ms, "band_sgm_ms": band_only_ms,
            "cnn_train_step_ms": train_ms, "cnn_train_batch": "16 x 270 x 480 cells",
            "banded_tile_fraction": statistics.mean(frac),
            "disagreement_mean": statistics.mean(dis), "disagreement_max": max(dis),
            "constant_centre_disagreement_mean": statistics.mean(const_dis)}


def _timed_ms(torch, fn, steps, flush, warmup=3):
    """Median CUDA-event time of fn on the current stream, L2 flushed before every call."""
    for _ in range(warmup):
        fn()
    ms = []
    for i in range(steps):
        flush.fill_(i & 0xff)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.median(ms)


def bench_full_hd(B, torch, synth, steps=10, cpu=True):
    """The whole path on the 1920x1080 road (seed 3: roll drawn in +-3 deg, five potholes),
    D = 128, 8 paths, SLIC with 1000 superpixels (compactness 10, 10 iterations, 1008 centres
    after the grid rounding) and the adaptive threshold: frames/s, the per-stage split from the
    library's events (captured graph, L2 flushed before each step), and the oracle's time for the
    same frame on one core."""
    sc = synth.road_1920x1080()
    left_np, right_np = synth.render(sc)
    H, W = left_np.shape
    D = 128
    ctx = B.Context(torch.cuda.current_device())
    B.pd_pipeline_config(ctx, True)
    model = B.RoadModel.make(*synth.true_model(sc))
    params = B.default_params(D=D, paths=8, slic_K=1000, slic_m=10.0, slic_iters=10)
    left, right = torch.from_numpy(left_np).cuda(), torch.from_numpy(right_np).cuda()
    outs = B.make_outputs(ctx, W, H)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        B.pd_run_pipeline(ctx, left, right, model, params, outs)
    torch.cuda.synchronize()
    B.pd_profile_enable(ctx, True)
    ms = []
    for i in range(steps):
        flush.fill_(i & 0xff)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        B.pd_run_pipeline(ctx, left, right, model, params, outs)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    prof = B.pd_profile_read(ctx)
    B.pd_profile_enable(ctx, False)
    calls = max(prof["calls"], 1)
    ctx.close()
    t = statistics.median(ms)
    stages = {k: prof[k] / calls for k in ("prep_ms", "aggregate_ms", "disparity_ms",
                                           "transform_ms", "superpixel_ms", "mask_ms")}
    sgm = stages["prep_ms"] + stages["aggregate_ms"] + stages["disparity_ms"]
    res = {"workload": "road_1920x1080 seed 3, D=128, 8 paths, SLIC 1000/10/10 (1008 centres), "
                       "threshold + mask + components; captured graph, L2 flushed per step",
           "ms_per_frame": t, "frames_per_s": 1e3 / t, "Mdisp_s": W * H * D / (t * 1e-3) / 1e6,
           "stage_ms": stages, "sgm_only_ms": sgm,
           "sgm_only_Mdisp_s": W * H * D / (sgm * 1e-3) / 1e6, "steps": steps}
    if cpu:
        import oracle
        oracle.lib()
        p = oracle.Params(D=D, paths=8, slic_K=1000, slic_m=10.0, slic_iters=10)
        t0 = time.perf_counter()
        oracle.pipeline(left_np, right_np, oracle.RoadModel.make(*synth.true_model(sc)), p)
        tc = time.perf_counter() - t0
        res["cpu_baseline"] = {"value": W * H * D / tc / 1e6, "unit": "Mdisp/s", "cores": 1,
                               "kind": "oracle", "frames_per_s": 1.0 / tc,
                               "sample": "one full 1920x1080 frame, whole oracle path, %.1f s" % tc}
    return res


def bench_pt(B, torch, synth, steps=10):
    """Sec. II-A at 1280x720 (the benchmark road): SGM (warp + cost + aggregation + disparity)
    with the row shifts of the road model at D = 128 (the benchmark's range), without them
    (kappa = 0, from the constant model f = delta_pt) at D = 128, which still holds the whole
    road's disparity (at most about 110 px here), and with them at D = 32, the residual range
    the shifts leave.  Times are CUDA-event medians with L2 flushed; accuracy against the
    generator's disparity over the pixels with u >= 127 (where every variant can have a result):
    the valid fraction, the mean |D1 - truth| of valid pixels and the share above 1 px."""
    import numpy as np
    sc = synth.road_1280x720()
    left_np, right_np = synth.render(sc)
    H, W = left_np.shape
    ctx = B.Context(torch.cuda.current_device())
    left, right = torch.from_numpy(left_np).cuda(), torch.from_numpy(right_np).cuda()
    gt = torch.from_numpy(synth.gt_disparity(sc).astype(np.float32)).cuda()[:, 127:]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    pt = B.RoadModel.make(*synth.true_model(sc))
    flat = B.RoadModel.make(1, (10.0, 0.0, 0.0), 0.0)   # f = delta_pt everywhere: kappa = 0
    out = {}
    for name, model, D in (("pt_d128", pt, 128), ("no_pt_d128", flat, 128), ("pt_d32", pt, 32)):
        p = B.default_params(D=D, paths=8)
        kap, d_int, D1 = B.pd_sgm(ctx, left, right, model, p)
        ms = _timed_ms(torch, lambda: B.pd_sgm(ctx, left, right, model, p, kap, d_int, D1), steps,
                       flush)
        v = D1[:, 127:]
        ok = v >= 0
        err = (v[ok] - gt[ok]).abs()
        out[name] = {"D": D, "ms": ms, "Mdisp_s": W * H * D / (ms * 1e-3) / 1e6,
                     "frames_per_s": 1e3 / ms, "kappa_range": [int(kap.min()), int(kap.max())],
                     "valid_fraction": ok.float().mean().item(),
                     "mean_abs_err_px": err.mean().item(),
                     "share_err_above_1px": (err > 1.0).float().mean().item()}
    ctx.close()
    out["workload"] = ("road_1280x720 seed 2, 8 paths: SGM with and without the perspective "
                       "transformation")
    return out


def main():
    args = parse()
    global W_, H_
    if args.size:
        W_, H_ = (int(x) for x in args.size.lower().split("x"))
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    from paper_2012_10802_gb300 import binding as B
    from paper_2012_10802_gb300 import synth

    torch.cuda.set_device(local)
    if args.int_peak:
        ctx = B.Context(local)
        with Clocks(local) as clk:
            rate, ipc = B.pd_int_rate(ctx)
        ctx.close()
        print(json.dumps({"pd_int_rate_lane_ops_per_s": rate, "T_lane_ops_per_s": rate / 1e12,
                          "thread_instr_per_clk_per_sm": ipc, "clocks": clk.summary()}))
        return
    if args.band_size:
        return band_only(B, torch, synth, args.band_size, args.steps, max(args.warmup, 3))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", rank=rank, world_size=world)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    # inputs: one synthetic pair per rank (independent frames: weak scaling, no collective)
    sc = synth.road_1280x720(seed=rank_seed(rank)) if (W_, H_) == (1280, 720) else \
        synth.road_scaled(W_, H_, seed=rank_seed(rank))
    left_np, right_np = synth.render(sc)
    model = B.RoadModel.make(*synth.true_model(sc))
    params = B.default_params()
    ctx = B.Context(local)
    B.pd_pipeline_config(ctx, not args.no_graph)  # replay the captured path (CUDA graph)
    left = torch.from_numpy(left_np).cuda()
    right = torch.from_numpy(right_np).cuda()
    outs = B.make_outputs(ctx, W_, H_)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    for _ in range(max(args.warmup, 3)):
        B.pd_run_pipeline(ctx, left, right, model, params, outs)
    torch.cuda.synchronize()

    # ---- timed region: device time of K steps, L2 flushed before each step
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    # only the two events around the aggregation are recorded in the timed steps (every event
    # drains the GPU between two stages); the full stage split comes from an untimed pass below
    B.pd_profile_enable(ctx, 2)
    for _ in range(2):                 # capture of the graph with those two events
        B.pd_run_pipeline(ctx, left, right, model, params, outs)
    torch.cuda.synchronize()
    B.pd_profile_read(ctx)
    with Clocks(local) as clk:
        barrier()
        t0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(i & 0xff)
            ev[i][0].record()
            B.pd_run_pipeline(ctx, left, right, model, params, outs)
            ev[i][1].record()
        barrier()
        wall = time.perf_counter() - t0
    prof_t = B.pd_profile_read(ctx)
    dev_ms = sum(a.elapsed_time(b) for a, b in ev)
    t_max = max_over_ranks(dev_ms, dist, "cuda")
    value = whole_job_mdisp(args.steps, world, W_, H_, D_, t_max)

    # ---- end to end through the public API: pinned host inputs in, the mask back out
    e2e = None
    if not args.no_e2e:
        lh = torch.from_numpy(left_np).pin_memory()
        rh = torch.from_numpy(right_np).pin_memory()
        mh = torch.empty((H_, W_), dtype=torch.uint8).pin_memory()
        ld, rd = torch.empty_like(left), torch.empty_like(right)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(2):
            ld.copy_(lh, non_blocking=True)
            rd.copy_(rh, non_blocking=True)
            B.pd_run_pipeline(ctx, ld, rd, model, params, outs)
            mh.copy_(outs[1]["mask"], non_blocking=True)
        barrier()
        e2e_local = 0.0
        for i in range(args.steps):
            flush.fill_((i + 7) & 0xff)            # L2 flushed before each step, as above
            e0.record()
            ld.copy_(lh, non_blocking=True)
            rd.copy_(rh, non_blocking=True)
            B.pd_run_pipeline(ctx, ld, rd, model, params, outs)
            mh.copy_(outs[1]["mask"], non_blocking=True)
            e1.record()
            e1.synchronize()
            e2e_local += e0.elapsed_time(e1)
        barrier()
        e2e_ms = max_over_ranks(e2e_local, dist, "cuda")
        e2e = {"value": whole_job_mdisp(args.steps, world, W_, H_, D_, e2e_ms),
               "unit": "Mdisp/s", "h2d_bytes_per_step": 2 * W_ * H_,
               "d2h_bytes_per_step": W_ * H_, "ms_per_step": e2e_ms / args.steps}
    # the e2e leg ran with the same two events as the device leg, so the two are comparable
    B.pd_profile_read(ctx)
    # the per-stage split: the same steps with every stage's events, untimed
    B.pd_profile_enable(ctx, True)
    for _ in range(2):
        B.pd_run_pipeline(ctx, left, right, model, params, outs)
    torch.cuda.synchronize()
    B.pd_profile_read(ctx)
    for i in range(args.steps):
        flush.fill_(i & 0xff)
        B.pd_run_pipeline(ctx, left, right, model, params, outs)
    prof = B.pd_profile_read(ctx)
    B.pd_profile_enable(ctx, False)

    if rank != 0:
        ctx.close()
        if dist:
            dist.destroy_process_group()
        return

    clocks = clk.summary()
    peaks = measured_peaks()
    calls = max(prof["calls"], 1)
    agg_ms = prof_t["aggregate_ms"] / max(prof_t["calls"], 1)   # over the timed steps
    sgm_ms = (prof["prep_ms"] + prof["aggregate_ms"] + prof["disparity_ms"]) / calls
    # the integer peak, measured now on this GPU (packed u16x2 DPX instructions, u16 lanes)
    int_rate, int_ipc = B.pd_int_rate(ctx)
    sm_mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
    pd_units = W_ * H_ * D_
    agg_ops = AGG_OPS_PER_UNIT * PATHS_ * pd_units
    path_ops = (AGG_OPS_PER_UNIT * PATHS_ + PATH_EXTRA_OPS) * pd_units
    path_bytes = PATH_BYTES_PER_PD * pd_units + PATH_BYTES_PER_PIXEL * W_ * H_
    hbm_peak = peaks.get("hbm_gbs") or 6800.0
    hbm_src = ("MEASURED_PEAKS.json hbm_gbs (measured)" if peaks.get("hbm_gbs")
               else "fallback 6800 GB/s (no MEASURED_PEAKS.json on this box)")

    def frac(ops, nbytes, ms):
        """max(bytes / HBM peak, ops / integer peak) over the measured time."""
        return max(nbytes / (hbm_peak * 1e9), ops / int_rate) / (ms * 1e-3)

    # this design's own traffic: one cost byte in and one L byte out per (pixel, disparity, path)
    design_bytes = 2 * PATHS_ * pd_units
    roofline = {"kernel": "k_aggregate (Eq. 8, all 8 directions, one launch)", "bound": "alu",
                "achieved": agg_ops / (agg_ms * 1e-3) / 1e12, "peak": int_rate / 1e12,
                "unit": "T int-ops/s (u16 lanes)", "frac": frac(agg_ops, path_bytes, agg_ms),
                "traffic": agg_traffic_record(),
                "algorithmic_ops_per_launch": agg_ops,
                "algorithmic_ops_per_unit": "8 per (pixel, disparity, path)",
                "algorithmic_bytes_per_launch": path_bytes, "avg_launch_ms": agg_ms,
                "peak_source": "measured live: pd_int_rate, packed u16x2 DPX, %.1f thread "
                               "instr/clk/SM x 2 lanes, at the run's clock" % int_ipc,
                "theoretical_peak": SMS * 128 * sm_mhz * 1e6 / 1e12,
                "theoretical_source": "152 SMs x 128 u16 lanes/clk x %.0f MHz (median SM clock)"
                                      % sm_mhz,
                "hbm_view": {"design_bytes_per_launch": design_bytes,
                             "design_GBs": design_bytes / (agg_ms * 1e-3) / 1e9,
                             "peak_GBs": hbm_peak, "peak_source": hbm_src,
                             "frac_of_hbm": design_bytes / (agg_ms * 1e-3) / 1e9 / hbm_peak},
                "path": {"scope": "SGM a1-a5: row shifts, warp, census, cost, aggregation, "
                                  "winner-take-all, sub-pixel, right view, LR check",
                         "bound": "alu", "ops": path_ops,
                         "ops_per_unit": "8R + 4 = %d per (pixel, disparity)"
                                         % (AGG_OPS_PER_UNIT * PATHS_ + PATH_EXTRA_OPS),
                         "bytes": path_bytes, "ms": sgm_ms,
                         "achieved": path_ops / (sgm_ms * 1e-3) / 1e12,
                         "frac": frac(path_ops, path_bytes, sgm_ms)}}

    # Sec. III accuracy of the benchmark frame against the generator's ground truth: disparity
    # D1 against the true disparity, mask against the pixels deeper than delta_PD
    acc = None
    if rank == 0:
        _, t = outs
        D4 = torch.from_numpy(synth.gt_disparity(sc).astype(np.float32)).cuda()
        gt = torch.from_numpy(synth.pothole_truth(sc, float(params.delta_pd)).astype(np.uint8)).cuda()
        acc = B.pd_accuracy(ctx, t["D1"], D4, t["mask"], gt)
        recs, ncomp = B.component_records(outs)
        acc["components"] = ncomp
        acc["kept_components"] = int(np.sum(recs["fake"] == 0)) if ncomp > 0 else 0

    batch = None
    if not args.no_batch and not args.size:
        batch = bench_batch(B, torch, synth)
    band_res = None
    if not args.no_band and not args.size:
        band_res = bench_band(B, torch, synth)
    stream_res = None
    if not args.no_stream and not args.size and rank == 0:
        stream_res = bench_stream(B, torch, synth, graph=not args.no_graph)
    full_hd = None
    if not args.no_full_hd and not args.size and rank == 0:
        full_hd = bench_full_hd(B, torch, synth, cpu=not args.no_cpu_baseline)
    pt_res = None
    if not args.no_pt_compare and not args.size and rank == 0:
        pt_res = bench_pt(B, torch, synth)

    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        oracle.lib()
        rows = 720
        t_cpu = oracle_pipeline_time(left_np, right_np, synth.true_model(sc), rows)
        cpu = {"value": W_ * rows * D_ / t_cpu / 1e6, "unit": "Mdisp/s", "cores": 1,
               "kind": "oracle", "sample": "one full 1280x720 frame, whole oracle path, %.1f s" % t_cpu}

    out = {
        "metric": METRIC, "value": value, "unit": "Mdisp/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u16+f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "W": W_, "H": H_, "D": D_, "paths": PATHS_,
                   "l2": "flushed before each timed step (256 MiB write)",
                   "cuda_graph": not args.no_graph,
                   "frames_per_s": args.steps * world / (t_max * 1e-3),
                   "sgm_only_ms": sgm_ms, "sgm_only_Mdisp_s": W_ * H_ * D_ / (sgm_ms * 1e-3) / 1e6,
                   "stage_ms": {k: prof[k] / calls for k in ("prep_ms", "aggregate_ms",
                                                            "disparity_ms", "transform_ms",
                                                            "superpixel_ms", "mask_ms")},
                   "wall_s": wall, "accuracy": acc, "batch64": batch, "band1080": band_res,
                   "stream720": stream_res, "full_hd": full_hd, "pt720": pt_res},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": prof_t["launches"], "clocks": clocks,
    }
    print(json.dumps(out))
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
