"""Python access to the C oracle (test infrastructure only).

The oracle is a plain single-threaded CPU restatement of the paper's steps (arXiv 2012.10802,
Sec. II).  Only the test suite, the smoke check and the benchmark's CPU-baseline leg use it; the
product path (the CUDA library and its binding) never imports this package.
"""
import ctypes as C
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        _declare(_lib)
    return _lib


class RoadModel(C.Structure):
    """Sec. II-A Eq. (3): f = a0 + a1 v' + a2 v'^2, v' the row coordinate after the inverse roll
    about the image centre."""
    _fields_ = [("order", C.c_int), ("a", C.c_double * 3), ("roll", C.c_double)]

    @staticmethod
    def make(order, a, roll):
        m = RoadModel()
        m.order = int(order)
        for i in range(3):
            m.a[i] = float(a[i]) if i < len(a) else 0.0
        m.roll = float(roll)
        return m

    def as_tuple(self):
        return self.order, tuple(self.a), self.roll


_P = C.c_void_p
_i = C.c_int
_d = C.c_double
_f = C.c_float


def _declare(L):
    sig = {
        "or_road_f": (_d, [C.POINTER(RoadModel), _i, _i, _d, _d]),
        "or_kappa": (None, [C.POINTER(RoadModel), _i, _i, _d, _P]),
        "or_warp": (None, [_P, _i, _i, _P, _P]),
        "or_census": (None, [_P, _i, _i, _P]),
        "or_cost": (None, [_P, _P, _i, _i, _i, _P]),
        "or_aggregate_dir": (None, [_P, _i, _i, _i, _i, _i, _i, _i, _P]),
        "or_aggregate_dir_raw": (None, [_P, _i, _i, _i, _i, _i, _i, _i, _P]),
        "or_aggregate": (None, [_P, _i, _i, _i, _i, _i, _i, _P]),
        "or_disparity": (None, [_P, _i, _i, _i, _P, _i, _P, _P]),
        "or_moments": (None, [_P, _i, _i, _P]),
        "or_e0min": (_d, [_P, _i, _i, _i, _d, _P]),
        "or_fit_road": (None, [_P, _i, _i, _i, C.POINTER(RoadModel)]),
        "or_transform": (None, [_P, _i, _i, C.POINTER(RoadModel), _f, _P]),
        "or_slic_grid": (_i, [_i, _i, _i, C.POINTER(_i), C.POINTER(_i)]),
        "or_slic": (_i, [_P, _i, _i, _i, _f, _i, _P, _P]),
        "or_superpixel_mean": (None, [_P, _P, _i, _i, _i, _P]),
        "or_threshold": (_i, [_P, _P, _i, _i, _f, _i, C.POINTER(_d), C.POINTER(_d), _P]),
        "or_mask": (None, [_P, _i, _i, _d, _P]),
        "or_fit_road_robust": (None, [_P, _i, _i, _i, _i, _f, C.POINTER(RoadModel)]),
        "or_ccl": (_i, [_P, _i, _i, _i, _P]),
        "or_components": (None, [_P, _P, _i, _i, _i, _P]),
        "or_band_windows": (None, [_P, _i, _i, _i, _i, _P, _P]),
        "or_aggregate_band": (None, [_P, _P, _P, _i, _i, _i, _i, _i, _i, _P]),
        "or_disparity_band": (None, [_P, _P, _P, _i, _i, _i, _P, _i, _P, _P]),
        "or_moment_sums_size": (C.c_size_t, []),
        "or_moments_export": (None, [_P, _P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ----------------------------------------------------------------------------- Sec. II-A

def road_f(model, W, H, u, v):
    return lib().or_road_f(C.byref(model), W, H, float(u), float(v))


def kappa(model, W, H, delta_pt):
    out = np.empty(H, np.int32)
    lib().or_kappa(C.byref(model), W, H, float(delta_pt), _ptr(out))
    return out


def warp(right, kap):
    right = _c(right, np.uint8)
    H, W = right.shape
    out = np.empty_like(right)
    lib().or_warp(_ptr(right), W, H, _ptr(_c(kap, np.int32)), _ptr(out))
    return out


# ----------------------------------------------------------------------------- Sec. II-B

def census(img):
    img = _c(img, np.uint8)
    H, W = img.shape
    out = np.empty((H, W), np.uint32)
    lib().or_census(_ptr(img), W, H, _ptr(out))
    return out


def cost(cl, cr, D):
    cl = _c(cl, np.uint32)
    cr = _c(cr, np.uint32)
    H, W = cl.shape
    out = np.empty((H, W, D), np.uint8)
    lib().or_cost(_ptr(cl), _ptr(cr), W, H, D, _ptr(out))
    return out


def aggregate_dir(cst, dx, dy, P1, P2):
    cst = _c(cst, np.uint8)
    H, W, D = cst.shape
    out = np.empty_like(cst)
    lib().or_aggregate_dir(_ptr(cst), W, H, D, dx, dy, P1, P2, _ptr(out))
    return out


def aggregate_dir_raw(cst, dx, dy, P1, P2):
    cst = _c(cst, np.uint8)
    H, W, D = cst.shape
    out = np.empty((H, W, D), np.int64)
    lib().or_aggregate_dir_raw(_ptr(cst), W, H, D, dx, dy, P1, P2, _ptr(out))
    return out


DIRECTIONS = [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1), (1, -1), (-1, 1)]


def aggregate(cst, paths, P1, P2):
    cst = _c(cst, np.uint8)
    H, W, D = cst.shape
    out = np.empty((H, W, D), np.uint16)
    lib().or_aggregate(_ptr(cst), W, H, D, paths, P1, P2, _ptr(out))
    return out


def disparity(S, kap, lr_tol):
    S = _c(S, np.uint16)
    H, W, D = S.shape
    d_int = np.empty((H, W), np.int16)
    D1 = np.empty((H, W), np.float32)
    lib().or_disparity(_ptr(S), W, H, D, _ptr(_c(kap, np.int32)), lr_tol, _ptr(d_int), _ptr(D1))
    return d_int, D1


# ----------------------------------------------------------------------------- Sec. II-C

class Moments:
    """Opaque exact moment sums (count, sum u~^i v~^j, sum q u~^i v~^j, sum q^2)."""

    def __init__(self, D1):
        D1 = _c(D1, np.float32)
        self.H, self.W = D1.shape
        self.buf = (C.c_char * lib().or_moment_sums_size())()
        lib().or_moments(_ptr(D1), self.W, self.H, self.buf)

    def export(self):
        raw = np.empty(46, np.int64)
        lib().or_moments_export(self.buf, _ptr(raw))
        vals = [int(raw[2 * i]) % (1 << 64) + (int(raw[2 * i + 1]) << 64) for i in range(23)]
        out = {"count": vals[0], "m": {}, "q": {}, "qq": vals[22]}
        k = 1
        for i in range(5):
            for j in range(5 - i):
                out["m"][(i, j)] = vals[k]
                k += 1
        for i in range(3):
            for j in range(3 - i):
                out["q"][(i, j)] = vals[k]
                k += 1
        return out


def moments(D1):
    return Moments(D1)


def e0min(mom, order, phi):
    beta = np.zeros(3, np.float64)
    e = lib().or_e0min(mom.buf, order, mom.W, mom.H, float(phi), _ptr(beta))
    return e, beta


def fit_road(mom, order):
    out = RoadModel()
    lib().or_fit_road(mom.buf, order, mom.W, mom.H, C.byref(out))
    return out


def transform(D1, model, delta_dt):
    D1 = _c(D1, np.float32)
    H, W = D1.shape
    out = np.empty_like(D1)
    lib().or_transform(_ptr(D1), W, H, C.byref(model), float(delta_dt), _ptr(out))
    return out


# ----------------------------------------------------------------------------- Sec. II-D/E

def slic_grid(W, H, K):
    nx, ny = _i(), _i()
    n = lib().or_slic_grid(W, H, K, C.byref(nx), C.byref(ny))
    return n, nx.value, ny.value


def slic(D2, K, m, iters):
    D2 = _c(D2, np.float32)
    H, W = D2.shape
    n, _, _ = slic_grid(W, H, K)
    labels = np.empty((H, W), np.int32)
    centres = np.empty((n, 3), np.float32)
    lib().or_slic(_ptr(D2), W, H, K, float(m), iters, _ptr(labels), _ptr(centres))
    return labels, centres


def superpixel_mean(D2, labels, nlabels):
    D2 = _c(D2, np.float32)
    H, W = D2.shape
    out = np.empty_like(D2)
    lib().or_superpixel_mean(_ptr(D2), _ptr(_c(labels, np.int32)), W, H, nlabels, _ptr(out))
    return out


def threshold(D2, D1, delta_pd, mode=0):
    D2 = _c(D2, np.float32)
    H, W = D2.shape
    E2 = np.empty(256, np.float64)
    tr, ts = _d(), _d()
    rc = lib().or_threshold(_ptr(D2), _ptr(_c(D1, np.float32)), W, H, float(delta_pd), mode,
                            C.byref(tr), C.byref(ts), _ptr(E2))
    return rc, tr.value, ts.value, E2


def mask(D3, t_s):
    D3 = _c(D3, np.float32)
    H, W = D3.shape
    out = np.empty((H, W), np.uint8)
    lib().or_mask(_ptr(D3), W, H, float(t_s), _ptr(out))
    return out


# ----------------------------------------------------------------------------- chains

@dataclass
class Params:
    """Method parameters (readings of the paper's constants; delta_pd = 2.36 is Sec. II-E's)."""
    D: int = 128
    paths: int = 8
    P1: int = 4
    P2: int = 32
    lr_tol: int = 1
    delta_pt: float = 10.0
    delta_dt: float = 16.0
    delta_pd: float = 2.36
    slic_K: int = 1000
    slic_m: float = 10.0
    slic_iters: int = 10
    model_order: int = 2
    threshold_mode: int = 0


def sgm(left, right, model, p: Params):
    """Sec. II-A/II-B: warp, census cost, aggregation, disparity.  Returns a dict of stages."""
    H, W = left.shape
    kap = kappa(model, W, H, p.delta_pt)
    rw = warp(right, kap)
    cl, cr = census(left), census(rw)
    cst = cost(cl, cr, p.D)
    S = aggregate(cst, p.paths, p.P1, p.P2)
    d_int, D1 = disparity(S, kap, p.lr_tol)
    return {"kappa": kap, "right_warped": rw, "census_left": cl, "census_right": cr,
            "cost": cst, "S": S, "d_int": d_int, "D1": D1}


def pipeline(left, right, model, p: Params, keep_volumes=False):
    """The whole path: SGM, Sec. II-C transform, Sec. II-D SLIC, Sec. II-E threshold and mask."""
    out = sgm(left, right, model, p)
    if not keep_volumes:
        out.pop("cost")
        out.pop("S")
    D1 = out["D1"]
    mom = moments(D1)
    fitted = fit_road(mom, p.model_order)
    D2 = transform(D1, fitted, p.delta_dt)
    labels, centres = slic(D2, p.slic_K, p.slic_m, p.slic_iters)
    D3 = superpixel_mean(D2, labels, centres.shape[0])
    rc, t_r, t_s, E2 = threshold(D2, D1, p.delta_pd, p.threshold_mode)
    out.update({"moments": mom, "fitted": fitted, "D2": D2, "labels": labels, "centres": centres,
                "D3": D3, "t_r": t_r, "t_s": t_s, "E2": E2,
                "mask": mask(D3, t_s)})
    return out


# ----------------------------------------------------------------------------- learned band

def band_windows(tile_lo, W, H, D, band=17):
    tl = _c(tile_lo, np.int16)
    lo = np.empty((H, W), np.int16)
    hi = np.empty((H, W), np.int16)
    lib().or_band_windows(_ptr(tl), W, H, D, band, _ptr(lo), _ptr(hi))
    return lo, hi


def aggregate_band(cst, lo, hi, paths, P1, P2):
    cst = _c(cst, np.uint8)
    H, W, D = cst.shape
    out = np.empty((H, W, D), np.uint16)
    lib().or_aggregate_band(_ptr(cst), _ptr(_c(lo, np.int16)), _ptr(_c(hi, np.int16)), W, H, D,
                            paths, P1, P2, _ptr(out))
    return out


def disparity_band(S, lo, hi, kap, lr_tol):
    S = _c(S, np.uint16)
    H, W, D = S.shape
    d_int = np.empty((H, W), np.int16)
    D1 = np.empty((H, W), np.float32)
    lib().or_disparity_band(_ptr(S), _ptr(_c(lo, np.int16)), _ptr(_c(hi, np.int16)), W, H, D,
                            _ptr(_c(kap, np.int32)), lr_tol, _ptr(d_int), _ptr(D1))
    return d_int, D1


def sgm_band(left, right, model, p: Params, tile_lo, band=17):
    """Sec. II-A/II-B with the disparity search restricted to per-tile windows."""
    H, W = left.shape
    kap = kappa(model, W, H, p.delta_pt)
    rw = warp(right, kap)
    cst = cost(census(left), census(rw), p.D)
    lo, hi = band_windows(tile_lo, W, H, p.D, band)
    S = aggregate_band(cst, lo, hi, p.paths, p.P1, p.P2)
    d_int, D1 = disparity_band(S, lo, hi, kap, p.lr_tol)
    return {"kappa": kap, "lo": lo, "hi": hi, "S": S, "d_int": d_int, "D1": D1}


# ----------------------------------------------------------------------------- Sec. II-E CCL

COMPONENT_FIELDS = ("label", "count", "umin", "vmin", "umax", "vmax", "sum_u", "sum_v",
                    "superpixels", "corner", "single", "fake")


def ccl(mask, conn=8):
    """Connected components of the mask: (labels [H][W] int32, number of components)."""
    m = _c(mask, np.uint8)
    H, W = m.shape
    labels = np.empty((H, W), np.int32)
    n = lib().or_ccl(_ptr(m), W, H, conn, _ptr(labels))
    return labels, n


def components(labels, sp_labels, n):
    """Per-component statistics and the fake-pothole flags, [n][12] int64 (COMPONENT_FIELDS)."""
    lab = _c(labels, np.int32)
    H, W = lab.shape
    out = np.zeros((max(n, 1), 12), np.int64)
    lib().or_components(_ptr(lab), _ptr(_c(sp_labels, np.int32)), W, H, n, _ptr(out))
    return out[:n]


# ----------------------------------------------------------------------------- Sec. III accuracy

ACCURACY_FIELDS = ("q", "e_p1", "e_p2", "e_p3", "e_r", "tp", "fp", "fn", "tn", "precision",
                   "recall", "accuracy", "fscore")


def accuracy(D1, D4, mask, gt_mask, eps=(1.0, 2.0, 3.0)):
    """Sec. III-A: the percentage of error pixels e_p = 100 / q * #{|D1 - D4| > eps} and the RMSE
    e_r = sqrt(sum (D1 - D4)^2 / q) over the q pixels with a disparity (D1 >= 0) and a finite
    ground truth D4; Sec. III-B: pixel precision, recall, accuracy and F-score of the pothole
    mask against the ground-truth mask.  Returns a dict with ACCURACY_FIELDS (NaN where a
    denominator is 0)."""
    D1 = np.asarray(D1, np.float64)
    D4 = np.asarray(D4, np.float64)
    valid = (D1 >= 0) & np.isfinite(D4)
    q = int(valid.sum())
    diff = D1[valid] - D4[valid]
    out = {"q": q}
    for k, e in enumerate(eps, 1):
        out["e_p%d" % k] = 100.0 * np.count_nonzero(np.abs(diff) > e) / q if q else float("nan")
    out["e_r"] = float(np.sqrt(np.sum(diff * diff) / q)) if q else float("nan")
    m = np.asarray(mask) != 0
    g = np.asarray(gt_mask) != 0
    tp, fp = int(np.sum(m & g)), int(np.sum(m & ~g))
    fn, tn = int(np.sum(~m & g)), int(np.sum(~m & ~g))
    out.update(tp=tp, fp=fp, fn=fn, tn=tn)
    out["precision"] = tp / (tp + fp) if tp + fp else float("nan")
    out["recall"] = tp / (tp + fn) if tp + fn else float("nan")
    out["accuracy"] = (tp + tn) / (tp + fp + fn + tn)
    p, r = out["precision"], out["recall"]
    out["fscore"] = 2 * p * r / (p + r) if tp else float("nan")
    return out


def fit_robust(D1, order, iters, tau):
    """Sec. II-C's fit followed by `iters` refits on the inliers within tau (reading R17)."""
    D1 = _c(D1, np.float32)
    H, W = D1.shape
    m = RoadModel()
    lib().or_fit_road_robust(_ptr(D1), W, H, order, iters, float(tau), C.byref(m))
    return m
