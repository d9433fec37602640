"""Thin Python binding of libpothole's C ABI (include/pothole.h), with the same call names.

Argument marshalling only: tensors are passed as device pointers with their sizes, outputs are
allocated with torch when not given, and every computation runs in the library's CUDA kernels.
There is no CPU fallback: if the library is missing or no GPU is present, calls raise.
"""
import ctypes as C
import os

import numpy as np

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpothole.so")

PD_OK, PD_ERR_INVALID_ARG, PD_ERR_OOM, PD_ERR_CUDA, PD_ERR_TIMEOUT, PD_ERR_UNSUPPORTED = range(6)
STATUS_NAMES = {0: "PD_OK", 1: "PD_ERR_INVALID_ARG", 2: "PD_ERR_OOM", 3: "PD_ERR_CUDA",
                4: "PD_ERR_TIMEOUT", 5: "PD_ERR_UNSUPPORTED"}


class PdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class RoadModel(C.Structure):
    _fields_ = [("order", C.c_int), ("a", C.c_double * 3), ("roll", C.c_double)]

    @staticmethod
    def make(order, a, roll):
        m = RoadModel()
        m.order = int(order)
        for i in range(3):
            m.a[i] = float(a[i]) if i < len(a) else 0.0
        m.roll = float(roll)
        return m

    @staticmethod
    def from_tensor(t):
        """Reads one pd_road_model from a uint8 tensor of its bytes (e.g. a device output)."""
        raw = bytes(t.detach().to("cpu").contiguous().numpy().tobytes())
        return RoadModel.from_buffer_copy(raw[:C.sizeof(RoadModel)])


class Params(C.Structure):
    _fields_ = [("D", C.c_int), ("paths", C.c_int), ("P1", C.c_int), ("P2", C.c_int),
                ("lr_tol", C.c_int), ("delta_pt", C.c_float), ("delta_dt", C.c_float),
                ("delta_pd", C.c_float), ("slic_K", C.c_int), ("slic_m", C.c_float),
                ("slic_iters", C.c_int), ("model_order", C.c_int), ("threshold_mode", C.c_int),
                ("fit_iters", C.c_int), ("fit_tau", C.c_float)]


class Outputs(C.Structure):
    _fields_ = [("kappa", C.c_void_p), ("d_int", C.c_void_p), ("D1", C.c_void_p),
                ("fitted", C.c_void_p), ("D2", C.c_void_p), ("labels", C.c_void_p),
                ("D3", C.c_void_p), ("thresholds", C.c_void_p), ("mask", C.c_void_p),
                ("components", C.c_void_p), ("comps", C.c_void_p), ("max_comps", C.c_int32),
                ("connectivity", C.c_int32), ("n_comps", C.c_void_p)]


class StageTimes(C.Structure):
    _fields_ = [("sgm_ms", C.c_float), ("transform_ms", C.c_float),
                ("superpixel_ms", C.c_float), ("mask_ms", C.c_float), ("total_ms", C.c_float)]


class Profile(C.Structure):
    _fields_ = [("calls", C.c_int), ("pad", C.c_int), ("launches", C.c_longlong),
                ("prep_ms", C.c_double), ("aggregate_ms", C.c_double),
                ("disparity_ms", C.c_double), ("transform_ms", C.c_double),
                ("superpixel_ms", C.c_double), ("mask_ms", C.c_double), ("total_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class Pair(C.Structure):
    _fields_ = [("left", C.c_void_p), ("right", C.c_void_p), ("W", C.c_int), ("H", C.c_int),
                ("pitch", C.c_size_t), ("D", C.c_int), ("pad", C.c_int), ("model", RoadModel),
                ("kappa", C.c_void_p), ("d_int", C.c_void_p), ("D1", C.c_void_p)]


_P, _i, _z, _f = C.c_void_p, C.c_int, C.c_size_t, C.c_float
SIGNATURES = {
    "pd_create": [C.POINTER(C.c_void_p), _i, _P],
    "pd_destroy": [_P],
    "pd_set_stream": [_P, _P],
    "pd_default_params": [C.POINTER(Params)],
    "pd_warp": [_P, _P, _i, _i, _z, C.POINTER(RoadModel), _f, _P, _P],
    "pd_census": [_P, _P, _i, _i, _z, _P],
    "pd_cost": [_P, _P, _P, _i, _i, _z, _i, _P],
    "pd_aggregate_dir": [_P, _P, _i, _i, _i, _i, _i, _i, _i, _P],
    "pd_aggregate": [_P, _P, _i, _i, _i, _i, _i, _i, _P],
    "pd_disparity": [_P, _P, _i, _i, _i, _P, _i, _P, _P],
    "pd_sgm": [_P, _P, _P, _i, _i, _z, C.POINTER(RoadModel), C.POINTER(Params), _P, _P, _P],
    "pd_sgm_band": [_P, _P, _P, _i, _i, _z, C.POINTER(RoadModel), C.POINTER(Params), _P, _i,
                    _P, _P, _P],
    "pd_cnn_create": [C.POINTER(C.c_void_p), _i, _i, _i, _i],
    "pd_cnn_destroy": [_P],
    "pd_cnn_set_params": [_P, _P, _P, _i],
    "pd_cnn_get_params": [_P, _P, _P, _i],
    "pd_cnn_forward": [_P, _P, _P, _i, _i, _i, _P],
    "pd_cnn_loss_grad": [_P, _P, _P, _P, _i, _i, _i, _P, _P],
    "pd_cnn_train_step": [_P, _P, _P, _P, _i, _i, _i, _f, _P],
    "pd_cnn_check": [_P, _P],
    "pd_cnn_probe_timeout": [_P, _P, C.c_longlong],
    "pd_band_input": [_P, _P, _P, _i, _i, _z, _P, _P],
    "pd_band_labels": [_P, _P, _P, _i, _i, _i, _P],
    "pd_band_tiles": [_P, _P, _i, _i, _i, _i, _P],
    "pd_sgm_learned": [_P, _P, _P, _P, _i, _i, _z, C.POINTER(RoadModel), C.POINTER(Params), _i,
                       _P, _P, _P, _P],
    "pd_components": [_P, _P, _P, _i, _i, _i, _P, _P, _i, _P],
    "pd_accuracy": [_P, _P, _P, _P, _P, _i, _i, _P, _P],
    "pd_transform_robust": [_P, _P, _i, _i, _i, _f, _i, _f, _P, _P],
    "pd_moments": [_P, _P, _i, _i, _P],
    "pd_transform": [_P, _P, _i, _i, _i, _f, _P, _P],
    "pd_superpixels": [_P, _P, _i, _i, _i, _f, _i, _P, _P, _P, C.POINTER(_i)],
    "pd_pothole_mask": [_P, _P, _P, _P, _i, _i, _f, _i, _P, _P, _P],
    "pd_run_pipeline": [_P, _P, _P, _i, _i, _z, C.POINTER(RoadModel), C.POINTER(Params),
                        C.POINTER(Outputs), C.POINTER(StageTimes)],
    "pd_transform_noalloc": [_P, _i, _i, _i, _f, _P, _P, _P],
    "pd_run_pipeline_dev": [_P, _P, _P, _i, _i, _z, _P, C.POINTER(Params), C.POINTER(Outputs),
                            C.POINTER(StageTimes)],
    "pd_batch_config": [_P, C.c_size_t, _i, _i],
    "pd_sgm_batch": [_P, C.POINTER(Pair), _i, C.POINTER(Params)],
    "pd_profile_enable": [_P, _i],
    "pd_pipeline_config": [_P, _i],
    "pd_profile_read": [_P, C.POINTER(Profile)],
    "pd_int_rate": [_P, _i, C.POINTER(C.c_double), C.POINTER(C.c_double)],
    "pd_cnn_save": [_P, _P, C.c_char_p, _P, C.c_size_t],
    "pd_cnn_load": [_P, _P, C.c_char_p, _P, C.c_size_t, C.POINTER(C.c_size_t)],
    "pd_cnn_checkpoint_info": [C.c_char_p, C.POINTER(C.c_int), C.POINTER(C.c_longlong),
                               C.POINTER(C.c_size_t)],
}
EXTRA = {"pd_last_error": (C.c_char_p, [_P]), "pd_workspace_bytes": (C.c_size_t, [_P]),
         "pd_cnn_num_params": (C.c_int, [])}

_lib = None


def lib():
    """Loads libpothole.so (built by __graft_entry__.build()); raises if it is absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libpothole.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = C.c_int
            fn.argtypes = args
        for name, (res, args) in EXTRA.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def default_params(**overrides):
    p = Params()
    lib().pd_default_params(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


class Context:
    """Owns one pd_ctx bound to a device and a stream (torch's current stream by default)."""

    def __init__(self, device=0, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("libpothole needs a CUDA GPU; none is available")
        self.device = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        h = C.c_void_p()
        st = lib().pd_create(C.byref(h), device, C.c_void_p(stream.cuda_stream))
        if st != PD_OK:
            raise PdError(st, "pd_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().pd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self.stream = stream
        self.check(lib().pd_set_stream(self.h, C.c_void_p(stream.cuda_stream)))

    def last_error(self):
        return lib().pd_last_error(self.h).decode()

    def workspace_bytes(self):
        return int(lib().pd_workspace_bytes(self.h))

    def check(self, st):
        if st != PD_OK:
            raise PdError(st, self.last_error())

    def empty(self, shape, dtype):
        return torch.empty(shape, dtype=dtype, device=self.device)


# ------------------------------------------------------------------ calls, C-ABI names

def pd_warp(ctx, right, model, delta_pt, right_warped=None, kappa=None, want_image=True):
    H, W = right.shape
    if kappa is None:
        kappa = ctx.empty((H,), torch.int32)
    if want_image and right_warped is None:
        right_warped = ctx.empty((H, W), torch.uint8)
    ctx.check(lib().pd_warp(ctx.h, _ptr(right), W, H, W, C.byref(model), float(delta_pt),
                            _ptr(right_warped) if want_image else None, _ptr(kappa)))
    return right_warped, kappa


def pd_census(ctx, img, codes=None):
    H, W = img.shape
    if codes is None:
        codes = ctx.empty((H, W), torch.int32)
    ctx.check(lib().pd_census(ctx.h, _ptr(img), W, H, W, _ptr(codes)))
    return codes


def pd_cost(ctx, left, right_warped, D, cost=None):
    H, W = left.shape
    if cost is None:
        cost = ctx.empty((H, W, D), torch.uint8)
    ctx.check(lib().pd_cost(ctx.h, _ptr(left), _ptr(right_warped), W, H, W, D, _ptr(cost)))
    return cost


def pd_aggregate_dir(ctx, cost, dx, dy, P1, P2, L=None):
    H, W, D = cost.shape
    if L is None:
        L = ctx.empty((H, W, D), torch.uint8)
    ctx.check(lib().pd_aggregate_dir(ctx.h, _ptr(cost), W, H, D, dx, dy, P1, P2, _ptr(L)))
    return L


def pd_aggregate(ctx, cost, paths, P1, P2, S=None):
    H, W, D = cost.shape
    if S is None:
        S = ctx.empty((H, W, D), torch.int16)
    ctx.check(lib().pd_aggregate(ctx.h, _ptr(cost), W, H, D, paths, P1, P2, _ptr(S)))
    return S


def pd_disparity(ctx, S, kappa, lr_tol, d_int=None, D1=None):
    H, W, D = S.shape
    if d_int is None:
        d_int = ctx.empty((H, W), torch.int16)
    if D1 is None:
        D1 = ctx.empty((H, W), torch.float32)
    ctx.check(lib().pd_disparity(ctx.h, _ptr(S), W, H, D, _ptr(kappa), lr_tol, _ptr(d_int),
                                 _ptr(D1)))
    return d_int, D1


def pd_sgm(ctx, left, right, model, params, kappa=None, d_int=None, D1=None):
    H, W = left.shape
    if kappa is None:
        kappa = ctx.empty((H,), torch.int32)
    if d_int is None:
        d_int = ctx.empty((H, W), torch.int16)
    if D1 is None:
        D1 = ctx.empty((H, W), torch.float32)
    ctx.check(lib().pd_sgm(ctx.h, _ptr(left), _ptr(right), W, H, W, C.byref(model),
                           C.byref(params), _ptr(kappa), _ptr(d_int), _ptr(D1)))
    return kappa, d_int, D1


def pd_sgm_band(ctx, left, right, model, params, tile_lo, band_width=17, kappa=None, d_int=None,
                D1=None):
    H, W = left.shape
    assert tile_lo.dtype == torch.int16 and tuple(tile_lo.shape) == ((H + 15) // 16, (W + 15) // 16)
    if kappa is None:
        kappa = ctx.empty((H,), torch.int32)
    if d_int is None:
        d_int = ctx.empty((H, W), torch.int16)
    if D1 is None:
        D1 = ctx.empty((H, W), torch.float32)
    ctx.check(lib().pd_sgm_band(ctx.h, _ptr(left), _ptr(right), W, H, W, C.byref(model),
                                C.byref(params), _ptr(tile_lo), band_width, _ptr(kappa),
                                _ptr(d_int), _ptr(D1)))
    return kappa, d_int, D1


COMPONENT_DTYPE = np.dtype([("label", np.int32), ("count", np.int32), ("umin", np.int32),
                            ("vmin", np.int32), ("umax", np.int32), ("vmax", np.int32),
                            ("sum_u", np.int64), ("sum_v", np.int64), ("superpixels", np.int32),
                            ("corner", np.int32), ("single", np.int32), ("fake", np.int32)])


def pd_components(ctx, mask, sp_labels, connectivity=8, max_comps=4096, labels=None):
    """Connected components of the mask: (labels [H][W] int32 device tensor, host array of
    component records (COMPONENT_DTYPE), component count).  Synchronises the stream."""
    H, W = mask.shape
    if labels is None:
        labels = ctx.empty((H, W), torch.int32)
    comps = ctx.empty((max(max_comps, 1) * COMPONENT_DTYPE.itemsize,), torch.uint8)
    n = ctx.empty((1,), torch.int32)
    ctx.check(lib().pd_components(ctx.h, _ptr(mask), _ptr(sp_labels), W, H, connectivity,
                                  _ptr(labels), _ptr(comps), max_comps, _ptr(n)))
    count = int(n.item())
    recs = comps.cpu().numpy().view(COMPONENT_DTYPE)[:max(0, min(count, max_comps))]
    return labels, recs, count


ACCURACY_FIELDS = ("q", "e_p1", "e_p2", "e_p3", "e_r", "tp", "fp", "fn", "tn", "precision",
                   "recall", "accuracy", "fscore")


def pd_accuracy(ctx, D1, D4, mask, gt_mask, eps=(1.0, 2.0, 3.0)):
    """Sec. III accuracy of D1 against D4 and of the mask against gt_mask: a dict of
    ACCURACY_FIELDS (synchronises the stream)."""
    H, W = D1.shape
    e = (C.c_float * 3)(*[float(x) for x in eps])
    out = ctx.empty((13,), torch.float64)
    ctx.check(lib().pd_accuracy(ctx.h, _ptr(D1), _ptr(D4), _ptr(mask), _ptr(gt_mask), W, H,
                                C.cast(e, C.c_void_p), _ptr(out)))
    vals = out.cpu().numpy()
    return {k: (int(v) if k in ("q", "tp", "fp", "fn", "tn") else float(v))
            for k, v in zip(ACCURACY_FIELDS, vals)}


class Cnn:
    """Owns one pd_cnn (the band network) sized for max_batch inputs of max_hd x max_wd cells."""

    def __init__(self, device=0, max_batch=1, max_hd=270, max_wd=480):
        if not torch.cuda.is_available():
            raise RuntimeError("libpothole needs a CUDA GPU; none is available")
        h = C.c_void_p()
        st = lib().pd_cnn_create(C.byref(h), device, max_batch, max_hd, max_wd)
        if st != PD_OK:
            raise PdError(st, "pd_cnn_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().pd_cnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pd_cnn_num_params():
    return int(lib().pd_cnn_num_params())


def pd_cnn_set_params(ctx, net, params):
    a = np.ascontiguousarray(params, dtype=np.float32)
    ctx.check(lib().pd_cnn_set_params(ctx.h, net.h, a.ctypes.data_as(C.c_void_p), a.size))


def pd_cnn_get_params(ctx, net):
    a = np.empty(pd_cnn_num_params(), np.float32)
    ctx.check(lib().pd_cnn_get_params(ctx.h, net.h, a.ctypes.data_as(C.c_void_p), a.size))
    return a


def pd_cnn_save(ctx, net, path, state=b""):
    """Writes the network's training checkpoint (parameters, Adam moments and step) with `state`,
    opaque caller bytes such as the training loop's generator state (see include/pothole.h)."""
    state = bytes(state)
    buf = C.create_string_buffer(state, len(state)) if state else None
    ctx.check(lib().pd_cnn_save(ctx.h, net.h, os.fsencode(path), buf, len(state)))


def pd_cnn_load(ctx, net, path):
    """Restores a checkpoint written by pd_cnn_save; returns the caller-state bytes saved with it."""
    n = C.c_size_t(0)
    info = pd_cnn_checkpoint_info(path)
    cap = info["state_bytes"] if info else 0
    buf = C.create_string_buffer(max(cap, 1))
    ctx.check(lib().pd_cnn_load(ctx.h, net.h, os.fsencode(path), buf, cap, C.byref(n)))
    return buf.raw[:n.value]


def pd_cnn_checkpoint_info(path):
    """Host-only check of a checkpoint file: {"n_params", "step", "state_bytes"}, or None when the
    file is missing or damaged (wrong magic, version, size or CRC)."""
    n, step, sb = C.c_int(0), C.c_longlong(0), C.c_size_t(0)
    st = lib().pd_cnn_checkpoint_info(os.fsencode(path), C.byref(n), C.byref(step), C.byref(sb))
    if st != PD_OK:
        return None
    return {"n_params": n.value, "step": step.value, "state_bytes": sb.value}


def _out_shape(Hd, Wd):
    return (Hd - 1) // 4 + 1, (Wd - 1) // 4 + 1


def pd_cnn_forward(ctx, net, x, out=None):
    """x: bf16 [B][Hd][Wd][2] (or [Hd][Wd][2]) on the device -> float [B][Ho][Wo][2]."""
    if x.dim() == 3:
        x = x.unsqueeze(0)
    assert x.dtype == torch.bfloat16 and x.is_contiguous()
    B, Hd, Wd, _ = x.shape
    Ho, Wo = _out_shape(Hd, Wd)
    if out is None:
        out = ctx.empty((B, Ho, Wo, 2), torch.float32)
    ctx.check(lib().pd_cnn_forward(ctx.h, net.h, _ptr(x), B, Hd, Wd, _ptr(out)))
    return out


def pd_cnn_check(ctx, net):
    """Synchronises; raises PdError (PD_ERR_TIMEOUT) if a tensor-core wait of the network ran out
    since the last check."""
    ctx.check(lib().pd_cnn_check(ctx.h, net.h))


def pd_cnn_probe_timeout(ctx, net, limit_cycles):
    ctx.check(lib().pd_cnn_probe_timeout(ctx.h, net.h, int(limit_cycles)))


def pd_cnn_loss_grad(ctx, net, x, targets):
    if x.dim() == 3:
        x = x.unsqueeze(0)
        targets = targets.unsqueeze(0)
    B, Hd, Wd, _ = x.shape
    loss = ctx.empty((1,), torch.float32)
    grad = ctx.empty((pd_cnn_num_params(),), torch.float32)
    ctx.check(lib().pd_cnn_loss_grad(ctx.h, net.h, _ptr(x), _ptr(targets), B, Hd, Wd, _ptr(loss),
                                     _ptr(grad)))
    return loss, grad


def pd_cnn_train_step(ctx, net, x, targets, lr, loss=None):
    if x.dim() == 3:
        x = x.unsqueeze(0)
        targets = targets.unsqueeze(0)
    B, Hd, Wd, _ = x.shape
    ctx.check(lib().pd_cnn_train_step(ctx.h, net.h, _ptr(x), _ptr(targets), B, Hd, Wd,
                                      float(lr), _ptr(loss)))
    return loss


def pd_band_input(ctx, left, right, kappa, x=None):
    H, W = left.shape
    if x is None:
        x = ctx.empty(((H + 3) // 4, (W + 3) // 4, 2), torch.bfloat16)
    ctx.check(lib().pd_band_input(ctx.h, _ptr(left), _ptr(right), W, H, W, _ptr(kappa), _ptr(x)))
    return x


def pd_band_labels(ctx, d_int, D1, D, targets=None):
    H, W = d_int.shape
    if targets is None:
        targets = ctx.empty(((H + 15) // 16, (W + 15) // 16, 4), torch.float32)
    ctx.check(lib().pd_band_labels(ctx.h, _ptr(d_int), _ptr(D1), W, H, D, _ptr(targets)))
    return targets


def pd_band_tiles(ctx, cnn_out, D, band_width=17, tile_lo=None):
    th, tw = cnn_out.shape[-3], cnn_out.shape[-2]
    if tile_lo is None:
        tile_lo = ctx.empty((th, tw), torch.int16)
    ctx.check(lib().pd_band_tiles(ctx.h, _ptr(cnn_out), th, tw, D, band_width, _ptr(tile_lo)))
    return tile_lo


def pd_sgm_learned(ctx, net, left, right, model, params, band_width=17, tile_lo=None, kappa=None,
                   d_int=None, D1=None):
    H, W = left.shape
    if tile_lo is None:
        tile_lo = ctx.empty(((H + 15) // 16, (W + 15) // 16), torch.int16)
    if kappa is None:
        kappa = ctx.empty((H,), torch.int32)
    if d_int is None:
        d_int = ctx.empty((H, W), torch.int16)
    if D1 is None:
        D1 = ctx.empty((H, W), torch.float32)
    ctx.check(lib().pd_sgm_learned(ctx.h, net.h, _ptr(left), _ptr(right), W, H, W, C.byref(model),
                                   C.byref(params), band_width, _ptr(tile_lo), _ptr(kappa),
                                   _ptr(d_int), _ptr(D1)))
    return tile_lo, kappa, d_int, D1


def pd_moments(ctx, D1, sums=None):
    H, W = D1.shape
    if sums is None:
        sums = ctx.empty((46,), torch.int64)
    ctx.check(lib().pd_moments(ctx.h, _ptr(D1), W, H, _ptr(sums)))
    return sums


def pd_transform(ctx, D1, order, delta_dt, fitted=None, D2=None):
    H, W = D1.shape
    if fitted is None:
        fitted = ctx.empty((C.sizeof(RoadModel),), torch.uint8)
    if D2 is None:
        D2 = ctx.empty((H, W), torch.float32)
    ctx.check(lib().pd_transform(ctx.h, _ptr(D1), W, H, order, float(delta_dt), _ptr(fitted),
                                 _ptr(D2)))
    return fitted, D2


def pd_transform_robust(ctx, D1, order, delta_dt, iters, tau, fitted=None, D2=None):
    H, W = D1.shape
    if fitted is None:
        fitted = ctx.empty((C.sizeof(RoadModel),), torch.uint8)
    if D2 is None:
        D2 = ctx.empty((H, W), torch.float32)
    ctx.check(lib().pd_transform_robust(ctx.h, _ptr(D1), W, H, order, float(delta_dt), int(iters),
                                        float(tau), _ptr(fitted), _ptr(D2)))
    return fitted, D2


def pd_superpixels(ctx, D2, K, m, iters, labels=None, D3=None, want_centres=False):
    H, W = D2.shape
    if labels is None:
        labels = ctx.empty((H, W), torch.int32)
    if D3 is None:
        D3 = ctx.empty((H, W), torch.float32)
    n = C.c_int(0)
    centres = ctx.empty((W * H * 3,), torch.float32) if want_centres else None
    ctx.check(lib().pd_superpixels(ctx.h, _ptr(D2), W, H, K, float(m), iters, _ptr(labels),
                                   _ptr(D3), _ptr(centres), C.byref(n)))
    if want_centres:
        centres = centres[:3 * n.value].view(n.value, 3)
    return labels, D3, centres, n.value


def pd_pothole_mask(ctx, D2, D1, D3, delta_pd, mode=0, mask=None, thresholds=None, E2=None):
    H, W = D2.shape
    if mask is None:
        mask = ctx.empty((H, W), torch.uint8)
    if thresholds is None:
        thresholds = ctx.empty((2,), torch.float64)
    ctx.check(lib().pd_pothole_mask(ctx.h, _ptr(D2), _ptr(D1), _ptr(D3), W, H, float(delta_pd),
                                    mode, _ptr(mask), _ptr(thresholds), _ptr(E2)))
    return mask, thresholds


def make_outputs(ctx, W, H, components=True, max_comps=4096, connectivity=8):
    """Allocates every pd_outputs buffer for a W x H frame (with the connected components unless
    components=False); returns (Outputs, dict of tensors)."""
    t = {"kappa": ctx.empty((H,), torch.int32), "d_int": ctx.empty((H, W), torch.int16),
         "D1": ctx.empty((H, W), torch.float32),
         "fitted": ctx.empty((C.sizeof(RoadModel),), torch.uint8),
         "D2": ctx.empty((H, W), torch.float32), "labels": ctx.empty((H, W), torch.int32),
         "D3": ctx.empty((H, W), torch.float32), "thresholds": ctx.empty((2,), torch.float64),
         "mask": ctx.empty((H, W), torch.uint8)}
    if components:
        t["components"] = ctx.empty((H, W), torch.int32)
        t["comps"] = ctx.empty((max(max_comps, 1) * COMPONENT_DTYPE.itemsize,), torch.uint8)
        t["n_comps"] = ctx.empty((1,), torch.int32)
    o = Outputs()
    for k, v in t.items():
        setattr(o, k, v.data_ptr())
    o.max_comps = max_comps if components else 0
    o.connectivity = connectivity
    return o, t


def component_records(outputs):
    """Host copy of the component records written by pd_run_pipeline (synchronises)."""
    _, t = outputs
    n = int(t["n_comps"].item())
    cap = t["comps"].numel() // COMPONENT_DTYPE.itemsize
    return t["comps"].cpu().numpy().view(COMPONENT_DTYPE)[:max(0, min(n, cap))], n


def pd_run_pipeline(ctx, left, right, model, params, outputs, times=False):
    H, W = left.shape
    o, _ = outputs
    st = StageTimes() if times else None
    ctx.check(lib().pd_run_pipeline(ctx.h, _ptr(left), _ptr(right), W, H, W, C.byref(model),
                                    C.byref(params), C.byref(o),
                                    C.byref(st) if times else None))
    return st


def pd_run_pipeline_dev(ctx, left, right, model_dev, params, outputs, times=False):
    """pd_run_pipeline with the road model in device memory (model_dev: a uint8 tensor holding one
    pd_road_model, e.g. outputs[1]["fitted"] of the previous frame, which may be updated in
    place)."""
    H, W = left.shape
    o, _ = outputs
    st = StageTimes() if times else None
    ctx.check(lib().pd_run_pipeline_dev(ctx.h, _ptr(left), _ptr(right), W, H, W, _ptr(model_dev),
                                        C.byref(params), C.byref(o),
                                        C.byref(st) if times else None))
    return st


def road_model_tensor(ctx, model):
    """One pd_road_model in device memory (uint8 tensor) from a host RoadModel."""
    raw = np.frombuffer(bytes(model), np.uint8).copy()
    return torch.from_numpy(raw).to(ctx.device)


def pd_profile_enable(ctx, on=True):
    """on: True / 1 every stage's events, 2 only the two around the aggregation, False / 0 off."""
    ctx.check(lib().pd_profile_enable(ctx.h, 2 if (on == 2 and on is not True) else (1 if on else 0)))


def pd_pipeline_config(ctx, use_graph=True):
    """Replays pd_run_pipeline / pd_run_pipeline_dev from a captured CUDA graph while the call is
    the captured one (see include/pothole.h)."""
    ctx.check(lib().pd_pipeline_config(ctx.h, 1 if use_graph else 0))


def pd_profile_read(ctx):
    p = Profile()
    ctx.check(lib().pd_profile_read(ctx.h, C.byref(p)))
    return p.as_dict()


def pd_int_rate(ctx, reps=4096):
    """Measured packed u16x2 DPX issue rate: (u16 lane-ops per second, thread instructions per
    SM clock)."""
    a, b = C.c_double(), C.c_double()
    ctx.check(lib().pd_int_rate(ctx.h, int(reps), C.byref(a), C.byref(b)))
    return a.value, b.value


def pd_transform_noalloc(D1, order, delta_dt, fitted, D2, stream=None):
    """The allocation-free transform: no context, fixed library scratch; outputs must be given."""
    H, W = D1.shape
    if stream is None:
        stream = torch.cuda.current_stream(D1.device)
    with torch.cuda.device(D1.device):     # the C side works on the current device
        return lib().pd_transform_noalloc(_ptr(D1), W, H, order, float(delta_dt), _ptr(fitted),
                                          _ptr(D2), C.c_void_p(stream.cuda_stream))


def pd_batch_config(ctx, scratch_budget_bytes=0, use_graph=False, autotune=True):
    ctx.check(lib().pd_batch_config(ctx.h, int(scratch_budget_bytes), 1 if use_graph else 0,
                                    1 if autotune else 0))


def make_batch(ctx, items):
    """items: list of (left, right, RoadModel, D).  Allocates the outputs; returns (Pair array,
    list of dicts with kappa / d_int / D1 tensors)."""
    arr = (Pair * len(items))()
    outs = []
    for k, (left, right, model, D) in enumerate(items):
        H, W = left.shape
        o = {"kappa": ctx.empty((H,), torch.int32), "d_int": ctx.empty((H, W), torch.int16),
             "D1": ctx.empty((H, W), torch.float32)}
        arr[k].left = left.data_ptr()
        arr[k].right = right.data_ptr()
        arr[k].W, arr[k].H, arr[k].pitch, arr[k].D = W, H, W, int(D)
        arr[k].model = model
        arr[k].kappa = o["kappa"].data_ptr()
        arr[k].d_int = o["d_int"].data_ptr()
        arr[k].D1 = o["D1"].data_ptr()
        outs.append(o)
    return arr, outs


def pd_sgm_batch(ctx, batch, params):
    arr, _ = batch
    ctx.check(lib().pd_sgm_batch(ctx.h, arr, len(arr), C.byref(params)))
