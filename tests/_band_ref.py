"""Layer-by-layer element-wise references for the band network's BF16 kernels
(test helper; imports only the oracle).

Each layer of the GPU network is checked on the GPU's own inputs to that
layer (read back with fbs_band_net_trace), so an error never propagates into
the next layer's check.  The reference is the FP64 network of
oracle/band_net.py with the same operands rounded to BF16 (weights, and the
exact BF16 inputs the kernel had); the kernels sum in FP32.  For a sum of n
terms t_i, in any order and with any rounding of the accumulator,

    |fl32(sum t_i) - sum t_i| <= gamma(n) * sum |t_i|,
    gamma(n) = n u / (1 - n u),  u = 2^-23

(twice the unit roundoff of round-to-nearest, which also covers truncation).
An element the kernel rounds to BF16 must therefore lie between the
roundings of the FP64 value minus and plus that bound; it must equal the
reference's rounding unless the FP64 value lies within the bound of a
rounding boundary (a midpoint between neighbouring BF16 values, or 0 under a
ReLU), where the kernel may round otherwise ("ambiguous").  A result other
than the reference's rounding inside the interval is a flip (counted); a
result outside it is a defect.  FP32
results (the network outputs, the weight gradients) must lie within
gamma(n) * sum|t_i| of the FP64 sum, plus one FP32 rounding.
"""

from __future__ import annotations

import numpy as np

from oracle import band_net as bn

U_ACC = 2.0 ** -23


def gamma(n):
    return n * U_ACC / (1.0 - n * U_ACC)


def rounding_check(got, z, eps, relu):
    """Compare BF16 results got with the FP64 values z (after a ReLU when
    relu).  The kernel's FP32 value lies in [z - eps, z + eps], and rounding
    is monotonic, so its BF16 result must lie in [RN(z - eps), RN(z + eps)];
    where that interval holds more than the rounding of z the element is
    ambiguous, and a result other than RN(z) inside it is a flip.  Returns
    (defects, flips, ambiguous) counts; defects must be 0."""
    z = np.asarray(z, np.float64)
    got = np.asarray(got, np.float64)
    eps = np.broadcast_to(np.asarray(eps, np.float64), z.shape)
    f = (lambda v: np.maximum(v, 0.0)) if relu else (lambda v: v)
    expect = bn.round_bf16(f(z))
    lo = bn.round_bf16(f(z - eps))
    hi = bn.round_bf16(f(z + eps))
    amb = lo != hi
    ok = (got >= lo) & (got <= hi)
    flip = ok & (got != expect)
    defect = ~ok
    if defect.any():
        for i in map(tuple, np.argwhere(defect)[:5]):
            print(f"  defect at {i}: fp64 {z[i]!r}, expected {expect[i]!r}, got {got[i]!r}, "
                  f"allowed [{lo[i]!r}, {hi[i]!r}]")
    return int(defect.sum()), int(flip.sum()), int(amb.sum())


def conv_with_scale(X, W, b):
    """conv(X; W) + b in FP64 and, per output, sum |terms| (bias included)."""
    return bn.conv3x3(X, W, b), bn.conv3x3(np.abs(X), np.abs(W), np.abs(b))


def conv_transpose_with_scale(G, W):
    """dL/dX of conv(X; W) given G = dL/d(conv output), and sum |terms|."""
    Xz = np.zeros(G.shape[:2] + (W.shape[2],))
    dX, _, _ = bn.conv3x3_backward(Xz, W, G)
    dXa, _, _ = bn.conv3x3_backward(Xz, np.abs(W), np.abs(G))
    return dX, dXa


def weight_grad_with_scale(X, G):
    """dW, db of sum(G * conv(X; W)) in FP64 and the sums of |terms|."""
    _, dW, db = bn.conv3x3_backward(X, np.zeros((3, 3, X.shape[2], G.shape[2])), G)
    _, dWa, dba = bn.conv3x3_backward(np.abs(X), np.zeros((3, 3, X.shape[2], G.shape[2])), np.abs(G))
    return dW, db, dWa, dba


def split_trace(acts, grads, Hq, Wq):
    """fbs_band_net_trace buffers -> (x0 [Hq][Wq][8], [Y1..Y5], O) and
    ([G1..G5], GO [Hq][Wq][8]) as float64 arrays."""
    P = Hq * Wq
    a = np.asarray(acts, np.float64)
    x0 = a[: P * 8].reshape(Hq, Wq, 8)
    o = P * 8
    ys = []
    for _ in range(5):
        ys.append(a[o: o + P * 32].reshape(Hq, Wq, 32))
        o += P * 32
    out = a[o: o + P * 2].reshape(Hq, Wq, 2)
    gs, go = None, None
    if grads is not None:
        g = np.asarray(grads, np.float64)
        gs, o = [], 0
        for _ in range(5):
            gs.append(g[o: o + P * 32].reshape(Hq, Wq, 32))
            o += P * 32
        go = g[o: o + P * 8].reshape(Hq, Wq, 8)
    return (x0, ys, out), (gs, go)
