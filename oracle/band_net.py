"""FP64 oracle of the band-proposal network (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this module; it shares no code with the CUDA path.

The network (the band form's reading of the paper's future-work idea,
Sec. V) maps the six quarter-resolution features of band_oracle.c to two
outputs per quarter pixel: o0, the correction of the coarse winner e* in
quarter-disparity units, and z, the logit of the confidence.  Six 3x3
convolutions with zero padding; ReLU after the first five:

    X_0 = features [Hq][Wq][6]
    Y_l = relu(conv(X_{l-1}; W_l) + b_l),  l = 1..5, 32 channels
    O   = conv(Y_5; W_6) + b_6,            2 channels (o0, z)
    conv(X; W)[y][x][o] = sum_{a,b in {-1,0,1}} sum_i X[y+a][x+b][i] W[a+1][b+1][i][o]
                          (X = 0 outside the image)

Loss over the N = Hq*Wq quarter pixels, with the predicted centre
c_i = 4 (e*_i + o0_i) in full-resolution disparities and the targets t_i, y_i
of band_oracle.c (reading B6):

    L = (1/N) sum_i [ y_i huber(c_i - t_i) + bce(z_i, y_i) ],
    huber(e) = e^2/2 for |e| <= 1, |e| - 1/2 otherwise,
    bce(z, y) = max(z, 0) - z y + log(1 + exp(-|z|)).

The centre term is weighted by the confidence target y (a constant of the
step): a block whose winners no band around the prediction can hold -- an
occlusion, a depth edge, the unmatched strip at the left border -- is left
to the full-range fallback instead of pulling the centre towards it.

Gradients are written out by the chain rule, layer by layer; the optimiser is
Adam (Kingma & Ba) with bias correction.  The flat parameter vector holds,
for l = 1..6, W_l as [3][3][Cin_l][Cout_l] followed by b_l [Cout_l].

``bf16=True`` rounds, to BF16 (round to nearest even), exactly the operands
that a BF16 tensor-core implementation holds in 16 bits -- the network input,
the weights, every hidden activation, and the gradients flowing backwards --
while every sum stays FP64.  That isolates the effect of the 16-bit operands
from the effect of the accumulation order.
"""

from __future__ import annotations

import numpy as np

N_FEATURES = 6
WIDTH = 32
N_OUT = 2
CIN = (N_FEATURES, WIDTH, WIDTH, WIDTH, WIDTH, WIDTH)
COUT = (WIDTH, WIDTH, WIDTH, WIDTH, WIDTH, N_OUT)
N_LAYERS = 6


def param_count() -> int:
    return sum(9 * ci * co + co for ci, co in zip(CIN, COUT))


def unpack(theta):
    """Flat vector -> list of (W [3][3][Cin][Cout], b [Cout]) views."""
    theta = np.asarray(theta, np.float64)
    out, o = [], 0
    for ci, co in zip(CIN, COUT):
        n = 9 * ci * co
        W = theta[o:o + n].reshape(3, 3, ci, co)
        o += n
        b = theta[o:o + co]
        o += co
        out.append((W, b))
    assert o == theta.size
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def round_bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.ascontiguousarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)


def _r(x, bf16):
    return round_bf16(x) if bf16 else x


def conv3x3(X, W, b):
    """conv(X; W) + b with zero padding.  X [H][W][Cin] -> [H][W][Cout]."""
    H, Wd, _ = X.shape
    Xp = np.zeros((H + 2, Wd + 2, X.shape[2]))
    Xp[1:H + 1, 1:Wd + 1] = X
    out = np.broadcast_to(b, (H, Wd, W.shape[3])).copy()
    for a in range(3):
        for c in range(3):
            out += Xp[a:a + H, c:c + Wd] @ W[a, c]
    return out


def conv3x3_backward(X, W, G):
    """Gradients of sum(G * conv(X; W)) w.r.t. X, W and b."""
    H, Wd, _ = X.shape
    Xp = np.zeros((H + 2, Wd + 2, X.shape[2]))
    Xp[1:H + 1, 1:Wd + 1] = X
    dW = np.empty_like(W)
    dXp = np.zeros_like(Xp)
    for a in range(3):
        for c in range(3):
            dW[a, c] = np.einsum("hwi,hwo->io", Xp[a:a + H, c:c + Wd], G)
            dXp[a:a + H, c:c + Wd] += G @ W[a, c].T
    return dXp[1:H + 1, 1:Wd + 1], dW, G.sum(axis=(0, 1))


def forward(theta, feat, bf16=False):
    """Network outputs O [Hq][Wq][2] and the layer inputs (for the backward pass)."""
    layers = unpack(theta)
    X = _r(np.asarray(feat, np.float64), bf16)
    acts = [X]
    for l, (W, b) in enumerate(layers):
        Z = conv3x3(X, _r(W, bf16), b)
        X = _r(np.maximum(Z, 0.0), bf16) if l < N_LAYERS - 1 else Z
        acts.append(X)
    return X, acts


def loss_and_output_grad(O, estar, t, y):
    """Loss L and dL/dO for outputs O [Hq][Wq][2]; t, y the targets."""
    o0, z = O[..., 0], O[..., 1]
    N = o0.size
    c = 4.0 * (np.asarray(estar, np.float64) + o0)
    y = np.asarray(y, np.float64)
    e = c - t
    ae = np.abs(e)
    huber = np.where(ae <= 1.0, 0.5 * e * e, ae - 0.5)
    bce = np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z)))
    L = float(((y * huber).sum() + bce.sum()) / N)
    dO = np.empty_like(O)
    dO[..., 0] = 4.0 * y * np.clip(e, -1.0, 1.0) / N
    dO[..., 1] = (1.0 / (1.0 + np.exp(-z)) - y) / N
    return L, dO


def backward(theta, acts, dO, bf16=False):
    """Gradient of the loss w.r.t. the flat parameter vector, given dL/dO."""
    layers = unpack(theta)
    grads = [None] * N_LAYERS
    G = _r(dO, bf16)
    for l in range(N_LAYERS - 1, -1, -1):
        W, _ = layers[l]
        dX, dW, db = conv3x3_backward(acts[l], _r(W, bf16), G)
        grads[l] = (dW, db)
        if l > 0:
            G = _r(dX * (acts[l] > 0.0), bf16)   # ReLU of layer l (acts[l] = Y_l)
    return pack(grads)


def adam_step(theta, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def centre_conf(O, estar):
    """Quarter-resolution centre 4 (e* + o0) and confidence sigmoid(z)."""
    return 4.0 * (np.asarray(estar, np.float64) + O[..., 0]), 1.0 / (1.0 + np.exp(-O[..., 1]))


def upsample(q, H, W):
    """Nearest-neighbour x4 upsampling of a quarter-resolution plane to H x W."""
    return np.asarray(q)[np.arange(H)[:, None] // 4, np.arange(W)[None, :] // 4]
