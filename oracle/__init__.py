"""FP64 CPU oracle for fast bilateral stereo (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package.  The product path (the CUDA library and its binding)
never does.  The C sources ``fbs_oracle.c`` (the method) and
``band_oracle.c`` (the band form's features, bands and targets) hold the
arithmetic; this module compiles them with gcc on first use (or from
``build()``) and wraps them with ctypes, plus the e_PEP metric of
Eq. (11)-(12).  The band network's FP64 oracle is ``band_net.py``.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "fbs_oracle.c"), os.path.join(_HERE, "band_oracle.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

COST_NCC = 0
COST_TAD = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no vector ISA flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(f) for f in _SRCS)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fno-fast-math",
                               "-ffp-contract=off", *_SRCS, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            Dd = ctypes.c_double
            lib.oracle_ncc.argtypes = [P, P, I, I, I, I, I, I]
            lib.oracle_ncc.restype = Dd
            lib.oracle_cost.argtypes = [P, P, I, I, I, I, I, I, I, Dd]
            lib.oracle_cost.restype = Dd
            lib.oracle_cost_volume.argtypes = [P, P, I, I, I, I, I, Dd, P]
            lib.oracle_weight.argtypes = [P, I, I, I, I, I, I, Dd, Dd]
            lib.oracle_weight.restype = Dd
            lib.oracle_aggregate.argtypes = [P, P, I, I, I, I, I, Dd, Dd, P]
            lib.oracle_aggregate_rows.argtypes = [P, I, P, I, I, I, I, I, Dd, Dd, I, I, P]
            lib.oracle_wta_subpixel.argtypes = [P, I, I, P, P]
            lib.oracle_fbs_rows.argtypes = [P, P, I, I, I, I, I, Dd, Dd, Dd, I, I, I, P, P, P]
            lib.oracle_fbs_rows.restype = I
            lib.oracle_fbs_points.argtypes = [P, P, I, I, I, I, I, Dd, Dd, Dd, I, I, P, P, P, P, P]
            lib.oracle_fbs_points.restype = I
            lib.oracle_fbs_right_rows.argtypes = [P, P, I, I, I, I, I, Dd, Dd, Dd, I, I, I, P, P, P]
            lib.oracle_fbs_right_rows.restype = I
            lib.oracle_lrc.argtypes = [P, P, I, I, P]
            lib.oracle_band_downsample.argtypes = [P, I, I, I, P]
            lib.oracle_band_features.argtypes = [P, P, I, I, I, I, P, P, P]
            lib.oracle_band_features.restype = I
            lib.oracle_band_limits.argtypes = [P, P, I, I, I, ctypes.c_float, P, P]
            lib.oracle_fbs_band_points.argtypes = [P, P, I, I, I, I, I, Dd, Dd, I, P, P, P, P, P, P, P]
            lib.oracle_fbs_band_points.restype = I
            lib.oracle_band_targets.argtypes = [P, P, I, I, I, I, P, P, P]
            lib.oracle_band_feature_points.argtypes = [P, P, I, I, I, I, Dd, P, P, Dd, P]
            lib.oracle_band_feature_points.restype = I
            _lib = lib
    return _lib


def _img(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    if a.ndim == 2:
        a = a[:, :, None]
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def ncc(left, right, u, v, d):
    """Eq. (1)-(3) at one (u, v, d); returns c in [-1, 1]."""
    L, R = _img(left), _img(right)
    H, W, C = L.shape
    return _load().oracle_ncc(_ptr(L), _ptr(R), H, W, C, u, v, d)


def cost_volume(left, right, D, mode=COST_NCC, tau=0.0):
    """Cost volume C[H][W][D] (float64)."""
    L, R = _img(left), _img(right)
    H, W, C = L.shape
    out = np.empty((H, W, D), np.float64)
    _load().oracle_cost_volume(_ptr(L), _ptr(R), H, W, C, D, mode, float(tau), _ptr(out))
    return out


def weight(guide, u, v, x, y, sigma_s, sigma_r):
    G = _img(guide)
    H, W, C = G.shape
    return _load().oracle_weight(_ptr(G), W, C, u, v, x, y, float(sigma_s), float(sigma_r))


def aggregate(cost, guide, radius, sigma_s, sigma_r):
    """Eq. (6): aggregated volume Agg[H][W][D] of a given cost volume."""
    G = _img(guide)
    H, W, C = G.shape
    cost = np.ascontiguousarray(cost, np.float64)
    D = cost.shape[2]
    assert cost.shape == (H, W, D)
    out = np.empty_like(cost)
    _load().oracle_aggregate(_ptr(cost), _ptr(G), H, W, C, D, int(radius), float(sigma_s),
                             float(sigma_r), _ptr(out))
    return out


def wta_subpixel(agg):
    """WTA (smallest d on ties) and Eq. (10) over the last axis of ``agg``."""
    agg = np.ascontiguousarray(agg, np.float64)
    D = agg.shape[-1]
    npix = agg.size // D
    di = np.empty(agg.shape[:-1], np.int32)
    ds = np.empty(agg.shape[:-1], np.float64)
    _load().oracle_wta_subpixel(_ptr(agg), npix, D, _ptr(di), _ptr(ds))
    return di, ds


def fbs(left, right, D, radius, sigma_s, sigma_r, tau=0.0, mode=COST_NCC, rows=None,
        want_agg=False):
    """The whole path.  ``rows`` = (y0, y1) restricts the output to a row band.

    Returns (d_int, d_sub) or (d_int, d_sub, agg) of the selected rows.
    """
    L, R = _img(left), _img(right)
    H, W, C = L.shape
    y0, y1 = rows if rows is not None else (0, H)
    n = (y1 - y0) * W
    di = np.empty((y1 - y0, W), np.int32)
    ds = np.empty((y1 - y0, W), np.float64)
    agg = np.empty((y1 - y0, W, D), np.float64) if want_agg else None
    rc = _load().oracle_fbs_rows(_ptr(L), _ptr(R), H, W, C, D, int(radius), float(sigma_s),
                                 float(sigma_r), float(tau), int(mode), y0, y1,
                                 _ptr(agg) if want_agg else None, _ptr(di), _ptr(ds))
    if rc != 0:
        raise MemoryError("oracle_fbs_rows could not allocate its cost rows")
    assert n == di.size
    return (di, ds, agg) if want_agg else (di, ds)


def fbs_right(left, right, D, radius, sigma_s, sigma_r, tau=0.0, mode=COST_NCC, rows=None, want_agg=False):
    """The right view: the right cost volume C_r(u, v, d) = C_l(u + d, v, d) (max cost
    where u + d >= W), aggregated with the right image as guide, WTA and Eq. (10)."""
    L, R = _img(left), _img(right)
    H, W, C = L.shape
    y0, y1 = rows if rows is not None else (0, H)
    di = np.empty((y1 - y0, W), np.int32)
    ds = np.empty((y1 - y0, W), np.float64)
    agg = np.empty((y1 - y0, W, D), np.float64) if want_agg else None
    rc = _load().oracle_fbs_right_rows(_ptr(L), _ptr(R), H, W, C, D, int(radius), float(sigma_s),
                                       float(sigma_r), float(tau), int(mode), y0, y1,
                                       _ptr(agg) if want_agg else None, _ptr(di), _ptr(ds))
    if rc != 0:
        raise MemoryError("oracle_fbs_right_rows could not allocate its cost rows")
    return (di, ds, agg) if want_agg else (di, ds)


def lrc(d_left, d_right):
    """Eq. (9): 1 where the left disparity is confirmed by the right map, else 0."""
    dl = np.ascontiguousarray(d_left, np.int32)
    dr = np.ascontiguousarray(d_right, np.int32)
    H, W = dl.shape
    out = np.empty((H, W), np.int32)
    _load().oracle_lrc(_ptr(dl), _ptr(dr), H, W, _ptr(out))
    return out


def fbs_points(left, right, D, radius, sigma_s, sigma_r, xs, ys, tau=0.0, mode=COST_NCC):
    """The whole path at isolated pixels; returns (d_int, d_sub, agg[n, D])."""
    L, R = _img(left), _img(right)
    H, W, C = L.shape
    xs = np.ascontiguousarray(xs, np.int32)
    ys = np.ascontiguousarray(ys, np.int32)
    n = xs.size
    di = np.empty(n, np.int32)
    ds = np.empty(n, np.float64)
    agg = np.empty((n, D), np.float64)
    rc = _load().oracle_fbs_points(_ptr(L), _ptr(R), H, W, C, D, int(radius), float(sigma_s),
                                   float(sigma_r), float(tau), int(mode), n, _ptr(xs), _ptr(ys),
                                   _ptr(agg), _ptr(di), _ptr(ds))
    if rc != 0:
        raise MemoryError("oracle_fbs_points could not allocate")
    return di, ds, agg


# ---------------------------------------------------------------------------
# Band form (readings B1-B6 of band_oracle.c)
# ---------------------------------------------------------------------------
def quarter_shape(H, W, D):
    return (H + 3) // 4, (W + 3) // 4, (D + 3) // 4


def band_downsample(img):
    """B1: quarter-resolution intensity (int32, Hq x Wq)."""
    I = _img(img)
    H, W, C = I.shape
    out = np.empty(((H + 3) // 4, (W + 3) // 4), np.int32)
    _load().oracle_band_downsample(_ptr(I), H, W, C, _ptr(out))
    return out


def band_features(left, right, D, with_gap=False):
    """B1-B3: features [Hq][Wq][6] (float64) and the coarse winner e* (int32);
    with_gap also returns, per quarter pixel, the second smallest minus the
    smallest coarse aggregated cost (the distance of the winner from a tie)."""
    L, R = _img(left), _img(right)
    H, W, C = L.shape
    Hq, Wq, _ = quarter_shape(H, W, D)
    feat = np.empty((Hq, Wq, 6), np.float64)
    est = np.empty((Hq, Wq), np.int32)
    gap = np.empty((Hq, Wq), np.float64)
    if _load().oracle_band_features(_ptr(L), _ptr(R), H, W, C, D, _ptr(feat), _ptr(est), _ptr(gap)) != 0:
        raise MemoryError("oracle_band_features could not allocate")
    return (feat, est, gap) if with_gap else (feat, est)


def band_limits(centre, conf, D, half_band, theta):
    """B4: per-pixel band [lo, hi] (int32 arrays of the input's shape)."""
    c = np.ascontiguousarray(centre, np.float32)
    k = np.ascontiguousarray(conf, np.float32)
    lo = np.empty(c.shape, np.int32)
    hi = np.empty(c.shape, np.int32)
    _load().oracle_band_limits(_ptr(c), _ptr(k), c.size, D, int(half_band), float(theta), _ptr(lo), _ptr(hi))
    return lo, hi


def fbs_band_points(left, right, D, radius, sigma_s, sigma_r, xs, ys, lo, hi):
    """B5 at isolated pixels with bands [lo_i, hi_i]; returns (d_int, d_sub, agg[n, D])
    with NaN outside each band."""
    L, R = _img(left), _img(right)
    H, W, C = L.shape
    xs = np.ascontiguousarray(xs, np.int32)
    ys = np.ascontiguousarray(ys, np.int32)
    lo = np.ascontiguousarray(lo, np.int32)
    hi = np.ascontiguousarray(hi, np.int32)
    n = xs.size
    di = np.empty(n, np.int32)
    ds = np.empty(n, np.float64)
    agg = np.empty((n, D), np.float64)
    rc = _load().oracle_fbs_band_points(_ptr(L), _ptr(R), H, W, C, D, int(radius), float(sigma_s),
                                        float(sigma_r), n, _ptr(xs), _ptr(ys), _ptr(lo), _ptr(hi),
                                        _ptr(agg), _ptr(di), _ptr(ds))
    if rc != 0:
        raise MemoryError("oracle_fbs_band_points could not allocate")
    return di, ds, agg


def band_targets(label_int, label_sub, D, half_band, centre_q):
    """B6: centre target t and confidence target y (both float64), Hq x Wq."""
    li = np.ascontiguousarray(label_int, np.int32)
    ls = np.ascontiguousarray(label_sub, np.float32)
    H, W = li.shape
    cq = np.ascontiguousarray(centre_q, np.float64)
    Hq, Wq = (H + 3) // 4, (W + 3) // 4
    assert cq.shape == (Hq, Wq)
    t = np.empty((Hq, Wq), np.float64)
    y = np.empty((Hq, Wq), np.float64)
    _load().oracle_band_targets(_ptr(li), _ptr(ls), H, W, D, int(half_band), _ptr(cq), _ptr(t), _ptr(y))
    return t, y


def band_feature_points(left, right, D, theta_m, tol=None):
    """B7: feature-point centre and confidence (float32, H x W).  With tol, also
    the pixels whose 5x5 quarter window holds a decision within tol of
    changing (a margin within tol of theta_m, or a winner within tol of a tie)."""
    L, R = _img(left), _img(right)
    H, W, C = L.shape
    c = np.empty((H, W), np.float32)
    k = np.empty((H, W), np.float32)
    amb = np.zeros((H, W), np.uint8)
    if _load().oracle_band_feature_points(_ptr(L), _ptr(R), H, W, C, D, float(theta_m), _ptr(c), _ptr(k),
                                          float(tol or 0.0), _ptr(amb)) != 0:
        raise MemoryError("oracle_band_feature_points could not allocate")
    return (c, k, amb.astype(bool)) if tol is not None else (c, k)


def e_pep(estimate, truth, eps, mask=None):
    """Eq. (11)-(12): percentage of pixels whose |estimate - truth| exceeds eps.

    ``mask`` (bool) selects the evaluated pixels; N is their count.
    """
    err = np.abs(np.asarray(estimate, np.float64) - np.asarray(truth, np.float64))
    bad = err > eps
    if mask is not None:
        bad = bad[mask]
    return 100.0 * float(np.count_nonzero(bad)) / max(1, bad.size)


def mde_per_s(W, H, D, seconds):
    """Eq. (13): millions of disparity evaluations per second."""
    return W * H * D / seconds * 1e-6
