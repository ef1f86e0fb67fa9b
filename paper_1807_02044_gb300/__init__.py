"""Python binding of libfbs, fast bilateral stereo on one GB300 GPU.

The binding only marshals arguments: every step of the path runs in the CUDA
kernels of ``libfbs.so`` (built by ``build.py``).  Functions carry the names
of the C ABI in ``include/fbs.h`` and ``include/fbs_band.h``.  Pointer arguments accept a CUDA tensor
(its ``data_ptr()``), a plain integer address, or None for NULL.  Streams
accept a ``torch.cuda.Stream``, a raw ``cudaStream_t`` integer, or None (the
context's own stream).  A non-OK status raises FBSError with the library's
message.  There is no CPU fallback: the library is loaded on first use, and
if it is missing that first call raises ImportError.  (Loading is deferred
only so that ``paper_1807_02044_gb300.build`` can be imported to build it.)
"""

from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfbs.so")

FBS_OK = 0
FBS_ERR_INVALID_ARG = 1
FBS_ERR_OOM = 2
FBS_ERR_CUDA = 3
FBS_ERR_TIMEOUT = 4
FBS_ERR_UNSUPPORTED = 5
STATUS_NAMES = {0: "FBS_OK", 1: "FBS_ERR_INVALID_ARG", 2: "FBS_ERR_OOM", 3: "FBS_ERR_CUDA",
                4: "FBS_ERR_TIMEOUT", 5: "FBS_ERR_UNSUPPORTED"}

FBS_COST_NCC = 0
FBS_COST_TAD = 1
FBS_PREC_F32 = 0
FBS_PREC_BF16 = 1
FBS_PREC_F16 = 2

FBS_KERNEL_COST = 0
FBS_KERNEL_AGG_F32 = 1
FBS_KERNEL_AGG_TC = 2
FBS_KERNEL_OTHER = 3
FBS_KERNEL_BATCH = 4
FBS_KERNEL_NET = 5
FBS_KERNEL_KINDS = 6
KERNEL_NAMES = {0: "cost_build", 1: "aggregate_f32", 2: "aggregate_tc", 3: "other", 4: "batch_graph",
                5: "band_net"}

FBS_BAND_FEATURES = 6
FBS_BAND_WIDTH = 32
FBS_BAND_LAYERS = 6

# Every function the header declares, with (restype, argtypes).
_P = ctypes.c_void_p
_I = ctypes.c_int
_F = ctypes.c_float
_Z = ctypes.c_size_t


class fbs_pair(ctypes.Structure):
    _fields_ = [("left", _P), ("right", _P), ("H", _I), ("W", _I), ("C", _I), ("D", _I), ("radius", _I),
                ("sigma_s", _F), ("sigma_r", _F), ("tau", _F), ("disp_int", _P), ("disp_subpix", _P)]


class fbs_options(ctypes.Structure):
    _fields_ = [("cost", _I), ("prec", _I), ("fused", _I), ("workspace_cap", _Z),
                ("autotune_cache_path", ctypes.c_char_p)]


SIGNATURES = {
    "fbs_default_options": (None, [ctypes.POINTER(fbs_options)]),
    "fbs_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(fbs_options), _I]),
    "fbs_destroy": (_I, [_P]),
    "fbs_set_options": (_I, [_P, ctypes.POINTER(fbs_options)]),
    "fbs_sync": (_I, [_P]),
    "fbs_set_wait_limit": (_I, [_P, ctypes.c_double]),
    "fbs_debug_fail_launches": (_I, [_P, _I, _I]),
    "fbs_last_error": (ctypes.c_char_p, [_P]),
    "fbs_compute_disparity": (_I, [_P, _P, _P, _I, _I, _I, _I, _I, _F, _F, _F, _P, _P, _P]),
    "fbs_compute_disparity_host": (_I, [_P, _P, _P, _I, _I, _I, _I, _I, _F, _F, _F, _P, _P]),
    "fbs_cost_volume": (_I, [_P, _P, _P, _I, _I, _I, _I, _F, _P, _P]),
    "fbs_compute_disparity_lr": (_I, [_P, _P, _P, _I, _I, _I, _I, _I, _F, _F, _F, _P, _P, _P, _P, _I, _P]),
    "fbs_aggregate": (_I, [_P, _P, _P, _I, _I, _I, _I, _I, _F, _F, _P, _P, _P, _P]),
    "fbs_compute_disparity_noalloc": (_I, [_P, _P, _P, _I, _I, _I, _I, _I, _F, _F, _F, _P, _P, _P]),
    "fbs_compute_disparity_batched": (_I, [_P, _I, _P, _P]),
    "fbs_batch_plan": (_I, [_P, _I, _P, ctypes.POINTER(_I)]),
    "fbs_batch_set_plan": (_I, [_P, _I, _P, _I]),
    "fbs_profile": (_I, [_P, _I]),
    "fbs_profile_read": (_I, [_P, _I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]),
    # fbs_band.h
    "fbs_band_net_param_count": (_Z, []),
    "fbs_band_net_init": (_I, [_P, ctypes.c_uint64]),
    "fbs_band_net_set_params": (_I, [_P, _P, _Z]),
    "fbs_band_net_get_params": (_I, [_P, _P, _Z]),
    "fbs_band_net_save": (_I, [_P, ctypes.c_char_p]),
    "fbs_band_net_load": (_I, [_P, ctypes.c_char_p]),
    "fbs_band_features": (_I, [_P, _P, _P, _I, _I, _I, _I, _P, _P, _P]),
    "fbs_band_net_forward": (_I, [_P, _P, _P, _I, _I, _I, _I, _P, _P, _P, _P]),
    "fbs_band_net_train_step": (_I, [_P, _P, _P, _I, _I, _I, _I, _P, _P, _I, _F, _P, _P, _P]),
    "fbs_band_limits": (_I, [_P, _P, _P, _I, _I, _I, _F, _P, _P, _P]),
    "fbs_band_net_trace": (_I, [_P, _P, _P, _P]),
    "fbs_band_feature_points": (_I, [_P, _P, _P, _I, _I, _I, _I, _F, _P, _P, _P]),
    "fbs_compute_disparity_banded": (_I, [_P, _P, _P, _P, _I, _F, _P]),
    "fbs_compute_disparity_learned": (_I, [_P, _P, _I, _F, _P]),
}


class FBSError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libfbs.so is not built ({LIB_PATH}); run paper_1807_02044_gb300.build.build() "
                          "or __graft_entry__.build() first. There is no CPU fallback.")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = _load()
    return _lib


def _addr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):          # numpy array (host entry point)
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


_CUDA_STREAM_LEGACY = 0x1   # cudaStreamLegacy: the device's legacy default stream


def _stream(s):
    """None -> NULL (the context's own stream).  A torch stream whose handle is
    0 is torch's legacy default stream; it is passed as cudaStreamLegacy so the
    library does not read it as NULL."""
    if s is None:
        return None
    if isinstance(s, int):
        return s
    h = s.cuda_stream
    return h if h else _CUDA_STREAM_LEGACY


def _check(ctx, status):
    if status != FBS_OK:
        msg = lib().fbs_last_error(ctx).decode() if ctx else ""
        raise FBSError(status, msg)


def fbs_default_options():
    o = fbs_options()
    lib().fbs_default_options(ctypes.byref(o))
    return o


def make_options(cost=FBS_COST_NCC, prec=FBS_PREC_F32, fused=0, workspace_cap=0):
    o = fbs_default_options()
    o.cost, o.prec, o.fused, o.workspace_cap = cost, prec, fused, workspace_cap
    return o


def fbs_create(options=None, device=0):
    ctx = _P()
    st = lib().fbs_create(ctypes.byref(ctx), ctypes.byref(options) if options is not None else None, device)
    if st != FBS_OK:
        raise FBSError(st, f"fbs_create(device={device}) failed")
    return ctx.value


def fbs_destroy(ctx):
    _check(None, lib().fbs_destroy(ctx))


def fbs_set_options(ctx, options):
    _check(ctx, lib().fbs_set_options(ctx, ctypes.byref(options)))


def fbs_sync(ctx):
    _check(ctx, lib().fbs_sync(ctx))


def fbs_set_wait_limit(ctx, seconds):
    _check(ctx, lib().fbs_set_wait_limit(ctx, float(seconds)))


def fbs_debug_fail_launches(ctx, cuda_error, count):
    _check(ctx, lib().fbs_debug_fail_launches(ctx, int(cuda_error), int(count)))


def fbs_last_error(ctx):
    return lib().fbs_last_error(ctx).decode()


def fbs_compute_disparity(ctx, left, right, H, W, C, D, radius, sigma_s, sigma_r, tau, disp_int, disp_subpix,
                          stream=None):
    _check(ctx, lib().fbs_compute_disparity(ctx, _addr(left), _addr(right), H, W, C, D, radius, sigma_s, sigma_r,
                                           tau, _addr(disp_int), _addr(disp_subpix), _stream(stream)))


def fbs_compute_disparity_host(ctx, left, right, H, W, C, D, radius, sigma_s, sigma_r, tau, disp_int,
                               disp_subpix):
    _check(ctx, lib().fbs_compute_disparity_host(ctx, _addr(left), _addr(right), H, W, C, D, radius, sigma_s,
                                                sigma_r, tau, _addr(disp_int), _addr(disp_subpix)))


FBS_NOALLOC_MAX_COST_BYTES = 32 * 1024 * 1024


def fbs_compute_disparity_noalloc(ctx, left, right, H, W, C, D, radius, sigma_s, sigma_r, tau, disp_int,
                                  disp_subpix, stream=None):
    """fbs_compute_disparity without device allocation: block statistics and
    cost volume go to the library's fixed static scratch, so
    H*W*(4*round_up(D,4)+20) bytes must not exceed FBS_NOALLOC_MAX_COST_BYTES."""
    _check(ctx, lib().fbs_compute_disparity_noalloc(ctx, _addr(left), _addr(right), H, W, C, D, radius, sigma_s,
                                                    sigma_r, tau, _addr(disp_int), _addr(disp_subpix),
                                                    _stream(stream)))


def fbs_compute_disparity_lr(ctx, left, right, H, W, C, D, radius, sigma_s, sigma_r, tau, disp_int, disp_subpix,
                             disp_int_right=None, disp_subpix_right=None, lrc=True, stream=None):
    """Both views and the left-right consistency check (Eq. (9)); rejected left
    pixels are -1 in both left outputs when lrc is true."""
    _check(ctx, lib().fbs_compute_disparity_lr(ctx, _addr(left), _addr(right), H, W, C, D, radius, sigma_s, sigma_r,
                                              tau, _addr(disp_int), _addr(disp_subpix), _addr(disp_int_right),
                                              _addr(disp_subpix_right), int(bool(lrc)), _stream(stream)))


def fbs_cost_volume(ctx, left, right, H, W, C, D, tau, cost_out, stream=None):
    _check(ctx, lib().fbs_cost_volume(ctx, _addr(left), _addr(right), H, W, C, D, tau, _addr(cost_out),
                                     _stream(stream)))


def fbs_aggregate(ctx, cost, guide, H, W, C, D, radius, sigma_s, sigma_r, agg_out, disp_int, disp_subpix,
                  stream=None):
    _check(ctx, lib().fbs_aggregate(ctx, _addr(cost), _addr(guide), H, W, C, D, radius, sigma_s, sigma_r,
                                   _addr(agg_out), _addr(disp_int), _addr(disp_subpix), _stream(stream)))


def make_pairs(pairs):
    """ctypes array of fbs_pair from dicts with keys left, right, H, W, C, D, radius,
    sigma_s, sigma_r, tau, disp_int, disp_subpix (tensors or addresses)."""
    arr = (fbs_pair * len(pairs))()
    for a, q in zip(arr, pairs):
        a.left, a.right = _addr(q["left"]), _addr(q["right"])
        a.H, a.W, a.C, a.D, a.radius = q["H"], q["W"], q["C"], q["D"], q["radius"]
        a.sigma_s, a.sigma_r, a.tau = q["sigma_s"], q["sigma_r"], q.get("tau", 0.0)
        a.disp_int, a.disp_subpix = _addr(q.get("disp_int")), _addr(q.get("disp_subpix"))
    return arr


def fbs_compute_disparity_batched(ctx, pairs, stream=None):
    """pairs: a ctypes fbs_pair array (see make_pairs) or a list of dicts."""
    arr = pairs if isinstance(pairs, ctypes.Array) else make_pairs(pairs)
    _check(ctx, lib().fbs_compute_disparity_batched(ctx, len(arr), ctypes.cast(arr, _P), _stream(stream)))


def fbs_batch_plan(ctx, pairs):
    arr = pairs if isinstance(pairs, ctypes.Array) else make_pairs(pairs)
    plan = _I()
    _check(ctx, lib().fbs_batch_plan(ctx, len(arr), ctypes.cast(arr, _P), ctypes.byref(plan)))
    return plan.value


def fbs_batch_set_plan(ctx, pairs, plan):
    arr = pairs if isinstance(pairs, ctypes.Array) else make_pairs(pairs)
    _check(ctx, lib().fbs_batch_set_plan(ctx, len(arr), ctypes.cast(arr, _P), int(plan)))


def fbs_profile(ctx, enable):
    _check(ctx, lib().fbs_profile(ctx, int(bool(enable))))


def fbs_profile_read(ctx, kind):
    """(summed device milliseconds, launch count) of one kernel kind."""
    ms = ctypes.c_double()
    n = ctypes.c_longlong()
    _check(ctx, lib().fbs_profile_read(ctx, kind, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


# ---- band form (fbs_band.h) ---------------------------------------------------
def default_band_net_path():
    """Weights of the band network trained by train_band_net.py for the
    1920x1080 RGB, D = 256, radius 9 workload (shipped with the package)."""
    return os.path.join(_HERE, "band_net_1920x1080_d256.bin")


def default_band_threshold():
    """Confidence threshold recorded with the shipped weights: the smallest one
    whose extra bad-pixel rate stayed under the training run's target on the
    held-out scenes."""
    import json
    with open(os.path.join(_HERE, "band_net_1920x1080_d256.json")) as f:
        return float(json.load(f)["threshold"])


def fbs_band_net_param_count():
    return int(lib().fbs_band_net_param_count())


def fbs_band_net_init(ctx, seed=0):
    _check(ctx, lib().fbs_band_net_init(ctx, int(seed)))


def fbs_band_net_set_params(ctx, params):
    """params: float32 numpy array of fbs_band_net_param_count() values (host)."""
    _check(ctx, lib().fbs_band_net_set_params(ctx, _addr(params), params.size))


def fbs_band_net_get_params(ctx, out):
    _check(ctx, lib().fbs_band_net_get_params(ctx, _addr(out), out.size))


def fbs_band_net_save(ctx, path):
    _check(ctx, lib().fbs_band_net_save(ctx, os.fsencode(path)))


def fbs_band_net_load(ctx, path):
    _check(ctx, lib().fbs_band_net_load(ctx, os.fsencode(path)))


def fbs_band_features(ctx, left, right, H, W, C, D, feat, estar, stream=None):
    _check(ctx, lib().fbs_band_features(ctx, _addr(left), _addr(right), H, W, C, D, _addr(feat), _addr(estar),
                                       _stream(stream)))


def fbs_band_net_forward(ctx, left, right, H, W, C, D, out_q, centre, conf, stream=None):
    _check(ctx, lib().fbs_band_net_forward(ctx, _addr(left), _addr(right), H, W, C, D, _addr(out_q),
                                          _addr(centre), _addr(conf), _stream(stream)))


def fbs_band_net_train_step(ctx, left, right, H, W, C, D, label_int, label_sub, half_band, lr, loss=None,
                            grad=None, stream=None):
    """loss: a 1-element float32 numpy array or None; grad: a float32 numpy array
    of fbs_band_net_param_count() values or None (both host)."""
    _check(ctx, lib().fbs_band_net_train_step(ctx, _addr(left), _addr(right), H, W, C, D, _addr(label_int),
                                             _addr(label_sub), half_band, lr, _addr(loss), _addr(grad),
                                             _stream(stream)))


def fbs_band_net_trace(ctx, acts=None, grads=None, stream=None):
    """Intermediate tensors of the last network call (see fbs_band.h): acts and
    grads are float32 CUDA tensors of P*(8+5*32+2) and P*(5*32+8) elements."""
    _check(ctx, lib().fbs_band_net_trace(ctx, _addr(acts), _addr(grads), _stream(stream)))


def fbs_band_feature_points(ctx, left, right, H, W, C, D, margin_threshold, centre, conf, stream=None):
    _check(ctx, lib().fbs_band_feature_points(ctx, _addr(left), _addr(right), H, W, C, D, margin_threshold,
                                             _addr(centre), _addr(conf), _stream(stream)))


def fbs_band_limits(ctx, centre, conf, n, D, half_band, conf_threshold, lo, hi, stream=None):
    _check(ctx, lib().fbs_band_limits(ctx, _addr(centre), _addr(conf), n, D, half_band, conf_threshold,
                                     _addr(lo), _addr(hi), _stream(stream)))


def fbs_compute_disparity_banded(ctx, pair, centre, conf, half_band, conf_threshold, stream=None):
    """pair: a dict as for make_pairs (or a one-element fbs_pair array)."""
    arr = pair if isinstance(pair, ctypes.Array) else make_pairs([pair])
    _check(ctx, lib().fbs_compute_disparity_banded(ctx, ctypes.cast(arr, _P), _addr(centre), _addr(conf),
                                                  half_band, conf_threshold, _stream(stream)))


def fbs_compute_disparity_learned(ctx, pair, half_band, conf_threshold, stream=None):
    arr = pair if isinstance(pair, ctypes.Array) else make_pairs([pair])
    _check(ctx, lib().fbs_compute_disparity_learned(ctx, ctypes.cast(arr, _P), half_band, conf_threshold,
                                                   _stream(stream)))


class Context:
    """Owning handle around fbs_create / fbs_destroy with tensor-level helpers."""

    def __init__(self, device=0, cost=FBS_COST_NCC, prec=FBS_PREC_F32, workspace_cap=0, autotune_cache_path=None):
        self.device = device
        self._opts = make_options(cost=cost, prec=prec, workspace_cap=workspace_cap)
        self._cache_path = autotune_cache_path.encode() if autotune_cache_path else None
        self._opts.autotune_cache_path = self._cache_path
        self.ctx = fbs_create(self._opts, device)

    def close(self):
        if self.ctx:
            fbs_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, cost=FBS_COST_NCC, prec=FBS_PREC_F32, workspace_cap=0):
        fbs_set_options(self.ctx, make_options(cost=cost, prec=prec, workspace_cap=workspace_cap))

    def compute_disparity(self, left, right, D, radius, sigma_s, sigma_r, tau=0.0, stream=None):
        """left, right: CUDA uint8 tensors (H, W, C) or (H, W).  Returns (disp_int, disp_subpix)."""
        import torch
        H, W = left.shape[0], left.shape[1]
        C = left.shape[2] if left.dim() == 3 else 1
        di = torch.empty((H, W), dtype=torch.int32, device=left.device)
        ds = torch.empty((H, W), dtype=torch.float32, device=left.device)
        if stream is None:
            stream = torch.cuda.current_stream(left.device)
        fbs_compute_disparity(self.ctx, left, right, H, W, C, D, radius, sigma_s, sigma_r, tau, di, ds, stream)
        return di, ds

    def cost_volume(self, left, right, D, tau=0.0, stream=None):
        import torch
        H, W = left.shape[0], left.shape[1]
        C = left.shape[2] if left.dim() == 3 else 1
        out = torch.empty((H, W, D), dtype=torch.float32, device=left.device)
        if stream is None:
            stream = torch.cuda.current_stream(left.device)
        fbs_cost_volume(self.ctx, left, right, H, W, C, D, tau, out, stream)
        return out

    def aggregate(self, cost, guide, radius, sigma_s, sigma_r, want_agg=True, stream=None):
        import torch
        H, W, D = cost.shape
        C = guide.shape[2] if guide.dim() == 3 else 1
        agg = torch.empty_like(cost) if want_agg else None
        di = torch.empty((H, W), dtype=torch.int32, device=cost.device)
        ds = torch.empty((H, W), dtype=torch.float32, device=cost.device)
        if stream is None:
            stream = torch.cuda.current_stream(cost.device)
        fbs_aggregate(self.ctx, cost, guide, H, W, C, D, radius, sigma_s, sigma_r, agg, di, ds, stream)
        return agg, di, ds
