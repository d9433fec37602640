"""Seeded synthetic stereo road scenes (inputs only; none of the method's steps live here).

The paper measures on KITTI stereo pairs and on its own pothole datasets; neither is available, so
every workload here is drawn from this generator instead.  A scene is a road whose ground-truth
disparity is quadratic in the row after a roll about the image centre (the road model family of
Sec. II-A), with elliptical potholes that lower the disparity with a cosine falloff.  The left image
is box-filtered uniform noise; the right image is the left one resampled through the ground-truth
disparity, plus Gaussian noise.

Used by the tests, the smoke check and the benchmark for both the CUDA path and the oracle.
"""
from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np


@dataclass
class Pothole:
    cu: float
    cv: float
    ax: float
    ay: float
    depth: float


@dataclass
class Scene:
    W: int
    H: int
    a: Tuple[float, float, float]
    roll: float  # radians
    potholes: List[Pothole] = field(default_factory=list)
    noise_sigma: float = 2.0
    seed: int = 0


def _rotated_row(W, H, u, v, roll):
    uc, vc = (W - 1) / 2.0, (H - 1) / 2.0
    return (v - vc) * np.cos(roll) - (u - uc) * np.sin(roll) + vc


def road_disparity(scene: Scene, u, v):
    """Ground-truth road disparity (no potholes) at real-valued (u, v)."""
    vp = _rotated_row(scene.W, scene.H, u, v, scene.roll)
    a0, a1, a2 = scene.a
    return a0 + a1 * vp + a2 * vp * vp


def pothole_offset(scene: Scene, u, v):
    off = np.zeros(np.broadcast(u, v).shape, np.float64)
    for p in scene.potholes:
        rho = np.sqrt(((u - p.cu) / p.ax) ** 2 + ((v - p.cv) / p.ay) ** 2)
        inside = rho < 1.0
        off = off - np.where(inside, p.depth * 0.5 * (1.0 + np.cos(np.pi * np.minimum(rho, 1.0))), 0.0)
    return off


def gt_disparity(scene: Scene, u=None, v=None):
    if u is None:
        v, u = np.mgrid[0:scene.H, 0:scene.W].astype(np.float64)
    return road_disparity(scene, u, v) + pothole_offset(scene, u, v)


def pothole_truth(scene: Scene, min_depth=0.0):
    """Boolean map of pixels whose pothole depth exceeds min_depth (for sanity checks only)."""
    v, u = np.mgrid[0:scene.H, 0:scene.W].astype(np.float64)
    return -pothole_offset(scene, u, v) > min_depth


def render(scene: Scene):
    """Returns (left, right) uint8 images of shape (H, W)."""
    rng = np.random.default_rng(scene.seed)
    W, H = scene.W, scene.H
    noise = rng.integers(0, 256, size=(H + 2, W + 2), dtype=np.int64)
    box = np.zeros((H, W), np.int64)
    for dy in range(3):
        for dx in range(3):
            box += noise[dy:dy + H, dx:dx + W]
    left = ((box + 4) // 9).astype(np.uint8)

    # right(x, v) = left(u, v) where x = u - d(u, v): solve for u by fixed-point iteration.
    v, x = np.mgrid[0:H, 0:W].astype(np.float64)
    u = x + gt_disparity(scene, x, v)
    for _ in range(3):
        u = x + gt_disparity(scene, u, v)
    u = np.clip(u, 0.0, W - 1.0)
    u0 = np.floor(u).astype(np.int64)
    u1 = np.minimum(u0 + 1, W - 1)
    t = u - u0
    rows = np.arange(H)[:, None]
    lf = left.astype(np.float64)
    val = (1.0 - t) * lf[rows, u0] + t * lf[rows, u1]
    val = val + rng.normal(0.0, scene.noise_sigma, size=(H, W))
    right = np.clip(np.rint(val), 0, 255).astype(np.uint8)
    return left, right


def _place_potholes(rng, W, H, a, roll, n, ax_rng, ay_rng, depth_rng, scale=1.0):
    holes = []
    probe = Scene(W, H, a, roll)
    attempts = 0
    while len(holes) < n and attempts < 1000:
        attempts += 1
        ax = rng.uniform(*ax_rng) * scale
        ay = rng.uniform(*ay_rng) * scale
        depth = rng.uniform(*depth_rng)
        cu = rng.uniform(ax, W - ax)
        cv = rng.uniform(H / 3.0 + ay, H - ay) if H / 3.0 + ay < H - ay else H * 2.0 / 3.0
        if road_disparity(probe, cu, cv) - depth < 2.0:
            continue
        holes.append(Pothole(cu, cv, ax, ay, depth))
    return holes


# ------------------------------------------------------------------------------- workloads
# Named by what they are: resolution, disparity range, paths.

def road_320x240(seed=1):
    """One pair 320x240: a = (5, 0.08, 1e-5), roll 1.5 deg, one 20x12 pothole 3 px deep."""
    s = Scene(320, 240, (5.0, 0.08, 1e-5), np.deg2rad(1.5), seed=seed)
    s.potholes = [Pothole(170.0, 180.0, 20.0, 12.0, 3.0)]
    return s


def road_1280x720(seed=2):
    """One pair 1280x720: a = (10, 0.12, 2e-5), roll 2 deg, three potholes (30-80 px, 2-8 px)."""
    rng = np.random.default_rng(seed + 7919)
    a = (10.0, 0.12, 2e-5)
    roll = np.deg2rad(2.0)
    s = Scene(1280, 720, a, roll, seed=seed)
    s.potholes = _place_potholes(rng, 1280, 720, a, roll, 3, (30, 80), (30, 80), (2, 8))
    return s


def road_1920x1080(seed=3):
    """One pair 1920x1080: the 720p road parameters, roll ~ U(+-3 deg), five potholes."""
    rng = np.random.default_rng(seed + 7919)
    a = (10.0, 0.12, 2e-5)
    roll = np.deg2rad(rng.uniform(-3.0, 3.0))
    s = Scene(1920, 1080, a, roll, seed=seed)
    s.potholes = _place_potholes(rng, 1920, 1080, a, roll, 5, (30, 80), (30, 80), (2, 8))
    return s


def road_scaled(W, H, seed, roll_deg=None, n_holes=3):
    """A road like the 720p one with disparity scaled to the image width (focal length in px
    grows with the width)."""
    rng = np.random.default_rng(seed + 7919)
    s = W / 1280.0
    a = (10.0 * s, 0.12, 2e-5 / s)
    roll = np.deg2rad(rng.uniform(-3.0, 3.0) if roll_deg is None else roll_deg)
    sc = Scene(W, H, a, roll, seed=seed)
    sc.potholes = _place_potholes(rng, W, H, a, roll, n_holes, (30, 80), (30, 80), (2, 8), scale=s)
    return sc


def mixed_batch(n=64, seed0=1000):
    """n pairs with resolutions from {640x480, 1280x720, 1920x1080} and residual disparity
    ranges from {32, 64, 128}; returns a list of (scene, D)."""
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed0 + i)
        W, H = [(640, 480), (1280, 720), (1920, 1080)][int(rng.integers(0, 3))]
        D = [32, 64, 128][int(rng.integers(0, 3))]
        out.append((road_scaled(W, H, seed0 + i), D))
    return out


def true_model(scene: Scene, order=2):
    """The scene's road model in the (order, a, roll) form of Sec. II-A Eq. (3)."""
    a = scene.a if order == 2 else (scene.a[0], scene.a[1], 0.0)
    return order, tuple(float(x) for x in a), float(scene.roll)


def render_torch(scene: Scene, device="cuda"):
    """The same scene model as render(), drawn on a CUDA device with torch's generator (seeded by
    the scene's seed): for producing many large training pairs quickly.  Returns (left, right)
    uint8 device tensors of shape (H, W).  The images follow render()'s recipe but not its
    random numbers."""
    import torch

    W, H = scene.W, scene.H
    g = torch.Generator(device=device)
    g.manual_seed(int(scene.seed))
    noise = torch.randint(0, 256, (H + 2, W + 2), generator=g, device=device, dtype=torch.int32)
    box = torch.zeros((H, W), dtype=torch.int32, device=device)
    for dy in range(3):
        for dx in range(3):
            box += noise[dy:dy + H, dx:dx + W]
    left = torch.div(box + 4, 9, rounding_mode="floor").to(torch.uint8)

    v = torch.arange(H, device=device, dtype=torch.float64)[:, None].expand(H, W)
    x = torch.arange(W, device=device, dtype=torch.float64)[None, :].expand(H, W)
    uc, vc = (W - 1) / 2.0, (H - 1) / 2.0
    cs, sn = float(np.cos(scene.roll)), float(np.sin(scene.roll))
    a0, a1, a2 = scene.a

    def disp(u):
        vp = (v - vc) * cs - (u - uc) * sn + vc
        d = a0 + a1 * vp + a2 * vp * vp
        for p in scene.potholes:
            rho = torch.sqrt(((u - p.cu) / p.ax) ** 2 + ((v - p.cv) / p.ay) ** 2)
            d = d - torch.where(rho < 1.0, p.depth * 0.5 * (1.0 + torch.cos(np.pi * torch.clamp(rho, max=1.0))),
                                torch.zeros_like(rho))
        return d

    u = x + disp(x)
    for _ in range(3):
        u = x + disp(u)
    u = torch.clamp(u, 0.0, W - 1.0)
    u0 = torch.floor(u).to(torch.int64)
    u1 = torch.clamp(u0 + 1, max=W - 1)
    t = u - u0
    lf = left.to(torch.float64)
    val = (1.0 - t) * torch.gather(lf, 1, u0) + t * torch.gather(lf, 1, u1)
    val = val + torch.randn((H, W), generator=g, device=device, dtype=torch.float64) * scene.noise_sigma
    right = torch.clamp(torch.round(val), 0, 255).to(torch.uint8)
    return left.contiguous(), right.contiguous()


def drive_sequence(W, H, n, seed, roll_step_deg=0.1, a0_step=0.05, hole_step=2.0):
    """n consecutive frames of a drive: the 720p-style road scaled to W x H whose roll turns by
    roll_step_deg and whose a0 grows by a0_step per frame, with the potholes moving down the image
    by hole_step rows per frame (each frame's noise drawn from its own seed)."""
    base = road_scaled(W, H, seed)
    frames = []
    for t in range(n):
        a = (base.a[0] + a0_step * t, base.a[1], base.a[2])
        holes = [Pothole(p.cu, p.cv + hole_step * t, p.ax, p.ay, p.depth) for p in base.potholes
                 if p.cv + hole_step * t + p.ay < H]
        frames.append(Scene(W, H, a, base.roll + np.deg2rad(roll_step_deg) * t, holes,
                            base.noise_sigma, seed * 1000 + t))
    return frames
