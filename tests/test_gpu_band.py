"""The learned band form on the GPU against the FP64 oracle.

Features and band limits are decided in the kernels' precision with the same
correctly rounded operations as the oracle, so they must match bit for bit.
The band-restricted path must match the oracle's band definition with the
tolerances of the plain path (integer winners identical except near ties,
subpixel within 1e-3).  The network runs on BF16 operands: every layer's
activations, outputs and gradients are compared element by element with the
FP64 network on the same BF16 operands, on the kernels' own inputs to the
layer, with the bounds derived below.
"""

import numpy as np
import pytest

from oracle import band_net as bn
from tests._compare import check_disparities

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fbs():
    from paper_1807_02044_gb300 import build as b
    b.build()
    import paper_1807_02044_gb300 as m
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rand_pair(seed, H, W, C=3, shift=5):
    rng = np.random.default_rng(seed)
    L = rng.integers(0, 256, size=(H, W, C)).astype(np.uint8)
    R = np.roll(L, -shift, axis=1)
    R = np.clip(R.astype(np.int16) + rng.integers(-6, 7, size=R.shape), 0, 255).astype(np.uint8)
    return L, R


# ---------------------------------------------------------------------------
# Features (against the FP64 oracle within the FP32 rounding bound), band
# limits (bit-exact)
# ---------------------------------------------------------------------------
# FP32 unit roundoff, and the bound on the kernels' coarse aggregated cost:
# K = 1 - num / sqrt(Vl Vr) from exact integers rounds the two conversions,
# the product, the square root, the conversion of num, the division and the
# subtraction (|c| <= 1, |K| <= 2): |dK| <= 6.5 u.  Kbar sums at most 25 such
# values (|K| <= 2) as row sums and a sum of row sums, then divides by the
# n >= 9 in-image taps: |dKbar| <= (4u 2n + 4u 2n + 6.5u n) / n + 2u = 24.5 u;
# the tests use 32 u.
U32 = 2.0 ** -24
TOL_KBAR = 32 * U32


def _gpu_features(fbs, L, R, D):
    H, W = L.shape[:2]
    C = L.shape[2] if L.ndim == 3 else 1
    Hq, Wq = (H + 3) // 4, (W + 3) // 4
    feat = torch.empty((Hq, Wq, 6), dtype=torch.float32, device="cuda")
    est = torch.empty((Hq, Wq), dtype=torch.int32, device="cuda")
    with fbs.Context(0) as ctx:
        fbs.fbs_band_features(ctx.ctx, _dev(L), _dev(R), H, W, C, D, feat, est)
        torch.cuda.synchronize()
        fbs.fbs_sync(ctx.ctx)
    return feat.cpu().numpy(), est.cpu().numpy()


@pytest.mark.parametrize("H,W,C,D", [(37, 45, 3, 40), (64, 200, 3, 128), (23, 530, 1, 64), (8, 8, 3, 4)])
def test_features_match_the_fp64_oracle(fbs, oracle_mod, H, W, C, D):
    """B1-B3 against the FP64 oracle: the coarse winner identical wherever the
    oracle's best and second best Kbar are more than 2 TOL_KBAR apart (at the
    others the kernel's winner must itself be within 2 TOL_KBAR of the best);
    f2 = Kbar(e*) within TOL_KBAR, the differences f3..f5 within 2 TOL_KBAR +
    2u, f0 within 2u, f1 = e*/Dq exact in FP32."""
    L, R = _rand_pair(H * W + D, H, W, C, shift=9)
    gf, ge = _gpu_features(fbs, L, R, D)
    rf, re, gap = oracle_mod.band_features(L, R, D, with_gap=True)
    Dq = (D + 3) // 4
    gf = gf.astype(np.float64)
    tie = gap <= 2 * TOL_KBAR
    assert np.array_equal(ge[~tie], re[~tie])
    assert np.all(np.abs(gf[..., 2] - rf[..., 2])[tie] <= 2 * TOL_KBAR)
    same = ge == re
    assert np.all(np.abs(gf[..., 2] - rf[..., 2])[same] <= TOL_KBAR)
    for k in (3, 4, 5):
        assert np.all(np.abs(gf[..., k] - rf[..., k])[same] <= 2 * TOL_KBAR + 2 * U32), k
    assert np.all(np.abs(gf[..., 0] - rf[..., 0]) <= 2 * U32)
    assert np.array_equal(gf[..., 1], (np.float32(1) * ge.astype(np.float32) / np.float32(Dq)).astype(np.float64))
    err = np.abs(gf[..., 2:] - rf[..., 2:])[same].max() if same.any() else 0.0
    print(f"{W}x{H} D={D}: {int(tie.sum())} near-tie quarter pixels of {tie.size}, "
          f"{int((~same).sum())} winners differ, max |d feature| {err:.2e} (bound {2 * TOL_KBAR + 2 * U32:.2e})")


def test_features_of_a_shift_by_four_k(fbs, oracle_mod):
    from synth import shifted_texture_pair
    H, W, D, k = 96, 256, 128, 7
    L, R = shifted_texture_pair(H, W, 3, 4 * k, seed=3)
    Hq, Wq, _ = oracle_mod.quarter_shape(H, W, D)
    est = torch.empty((Hq, Wq), dtype=torch.int32, device="cuda")
    with fbs.Context(0) as ctx:
        fbs.fbs_band_features(ctx.ctx, _dev(L), _dev(R), H, W, 3, D, None, est)
        torch.cuda.synchronize()
    assert np.all(est.cpu().numpy()[3:-3, k + 3:-3] == k)


def test_band_limits_bit_exact(fbs, oracle_mod):
    rng = np.random.default_rng(4)
    n, D, h, th = 5000, 100, 8, 0.5
    c = rng.uniform(-20, 120, n).astype(np.float32)
    c[:50] = np.floor(c[:50]) + 0.5          # exact halves
    c[50:60] = [np.nan, np.inf, -np.inf, 3e38, -3e38, 0.0, -0.0, 99.49, 99.5, 1e-30]
    k = rng.uniform(0, 1, n).astype(np.float32)
    k[60:70] = [np.nan, th, np.nextafter(np.float32(th), np.float32(0)), 1, 0, np.inf, -np.inf, 0.5, 0.5, 0.5]
    lo = torch.empty(n, dtype=torch.int32, device="cuda")
    hi = torch.empty(n, dtype=torch.int32, device="cuda")
    with fbs.Context(0) as ctx:
        fbs.fbs_band_limits(ctx.ctx, _dev(c), _dev(k), n, D, h, th, lo, hi)
        torch.cuda.synchronize()
    rlo, rhi = oracle_mod.band_limits(c, k, D, h, th)
    assert np.array_equal(lo.cpu().numpy(), rlo)
    assert np.array_equal(hi.cpu().numpy(), rhi)


# ---------------------------------------------------------------------------
# Band-restricted path
# ---------------------------------------------------------------------------
def _banded(fbs, ctx, L, R, D, r, ss, sr, centre, conf, h, th):
    H, W, C = L.shape
    di = torch.empty((H, W), dtype=torch.int32, device="cuda")
    ds = torch.empty((H, W), dtype=torch.float32, device="cuda")
    pair = dict(left=_dev(L), right=_dev(R), H=H, W=W, C=C, D=D, radius=r, sigma_s=ss, sigma_r=sr, tau=0.0,
                disp_int=di, disp_subpix=ds)
    fbs.fbs_compute_disparity_banded(ctx.ctx, pair, _dev(centre), _dev(conf), h, th)
    torch.cuda.synchronize()
    fbs.fbs_sync(ctx.ctx)
    return di.cpu().numpy(), ds.cpu().numpy()


def _check_band(di, ds, ragg, rdi, rds, lo, hi):
    """The plain path's rules with each pixel's candidates limited to its band
    (the oracle leaves NaN outside the band; +inf keeps them out of every
    minimum, and makes Eq. (10) at a band end count as not checkable)."""
    assert np.all((di >= lo) & (di <= hi))
    a = np.where(np.isnan(ragg), np.inf, ragg)
    return check_disparities(di, ds, a, rdi, rds, 2.0)


@pytest.mark.parametrize("H,W,D,r,h", [(29, 70, 48, 3, 4), (40, 131, 96, 5, 8), (17, 33, 20, 2, 3)])
def test_banded_matches_oracle_whole_frame(fbs, oracle_mod, H, W, D, r, h):
    L, R = _rand_pair(3 * H + W, H, W, 3, shift=6)
    rng = np.random.default_rng(H + D)
    centre = rng.uniform(-5, D + 5, (H, W)).astype(np.float32)
    centre[: H // 2] = 6.0 + rng.uniform(-3, 3, (H // 2, W)).astype(np.float32)   # bands around the truth
    conf = rng.uniform(0, 1, (H, W)).astype(np.float32)
    th = 0.3
    with fbs.Context(0) as ctx:
        di, ds = _banded(fbs, ctx, L, R, D, r, float(r), 12.0, centre, conf, h, th)
    lo, hi = oracle_mod.band_limits(centre.ravel(), conf.ravel(), D, h, th)
    ys, xs = np.mgrid[0:H, 0:W]
    rdi, rds, ragg = oracle_mod.fbs_band_points(L, R, D, r, float(r), 12.0, xs.ravel(), ys.ravel(), lo, hi)
    _check_band(di.ravel(), ds.ravel(), ragg, rdi, rds, lo, hi)


def test_banded_with_no_confident_pixel_equals_the_plain_path_bitwise(fbs):
    H, W, D, r = 45, 170, 72, 4
    L, R = _rand_pair(9, H, W, 3, shift=11)
    centre = np.full((H, W), 20.0, np.float32)
    conf = np.zeros((H, W), np.float32)
    with fbs.Context(0) as ctx:
        di, ds = _banded(fbs, ctx, L, R, D, r, 4.0, 12.0, centre, conf, 8, 0.5)
        pdi, pds = ctx.compute_disparity(_dev(L), _dev(R), D, r, 4.0, 12.0)
        torch.cuda.synchronize()
    assert np.array_equal(di, pdi.cpu().numpy())
    assert np.array_equal(ds.view(np.uint32), pds.cpu().numpy().view(np.uint32))


def test_banded_full_size_sampled(fbs, oracle_mod):
    """1920x1080 RGB, D=256, radius 9, half band 8: bands around a coarse
    estimate with 20% of the pixels falling back to the full range; 200
    sampled pixels against the oracle."""
    from synth import make_pair
    p = make_pair("rgb1920x1080_d256_r9", 1)
    rng = np.random.default_rng(2)
    centre = (p.gt + rng.normal(0, 3, p.gt.shape)).astype(np.float32)
    conf = (rng.uniform(0, 1, p.gt.shape) > 0.2).astype(np.float32)
    with fbs.Context(0) as ctx:
        di, ds = _banded(fbs, ctx, p.left, p.right, p.D, p.radius, p.sigma_s, p.sigma_r, centre, conf, 8, 0.5)
    ys = rng.integers(0, p.H, 200)
    xs = rng.integers(0, p.W, 200)
    lo, hi = oracle_mod.band_limits(centre[ys, xs], conf[ys, xs], p.D, 8, 0.5)
    rdi, rds, ragg = oracle_mod.fbs_band_points(p.left, p.right, p.D, p.radius, p.sigma_s, p.sigma_r, xs, ys,
                                                lo, hi)
    _check_band(di[ys, xs], ds[ys, xs], ragg, rdi, rds, lo, hi)


# ---------------------------------------------------------------------------
# Network: every layer element by element, on the kernels' own inputs
# ---------------------------------------------------------------------------
# fbs_band_net_trace reads back the kernels' input, hidden activations,
# outputs and backward gradients.  Each layer is checked on the GPU's own
# inputs to it against the FP64 network with the same BF16 operands
# (tests/_band_ref.py): a hidden activation or a backward gradient must equal
# the BF16 rounding of the FP64 value, except at "ambiguous" elements whose
# FP64 value lies within the FP32 accumulation bound gamma(n) * sum|terms| of a
# rounding boundary (n = 9 Cin + 1 terms of a convolution, 9 Cout of a data
# gradient); there only the other rounding is allowed (a "flip", counted).
# The outputs and the weight gradients (FP32 results) must lie within
# gamma(n) * sum|terms| of the FP64 sum (n = 9 Cin + 1, or the number of
# quarter pixels for a weight gradient) plus one FP32 rounding.
#
# End to end, against the unrounded FP64 network, the effect of the BF16
# operands is reported and bounded loosely (unit roundoff u = 2^-9; six forward
# layers compound to ~6-12u in norm for the outputs; a weight gradient passes
# through up to eleven roundings and the ReLU masks of the forward pass).
OUT_TOL = 0.03
GRAD_TOL = 0.15


def _params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    th = np.zeros(bn.param_count())
    o = 0
    for ci, co in zip(bn.CIN, bn.COUT):
        n = 9 * ci * co
        th[o:o + n] = rng.standard_normal(n) * np.sqrt(2.0 / (9 * ci)) * scale
        th[o + n:o + n + co] = rng.uniform(-0.1, 0.1, co)
        o += n + co
    return th.astype(np.float32)


def test_param_layout_matches_the_oracle(fbs):
    assert fbs.fbs_band_net_param_count() == bn.param_count()


def _trace_sizes(Hq, Wq):
    P = Hq * Wq
    return P * (8 + 5 * 32 + 2), P * (5 * 32 + 8)


@pytest.mark.parametrize("H,W,D", [(96, 160, 64), (53, 77, 40)])
def test_forward_layers_match_elementwise(fbs, oracle_mod, H, W, D):
    from tests import _band_ref as br
    L, R = _rand_pair(H + W, H, W, 3, shift=12)
    theta = _params(1)
    Hq, Wq, _ = oracle_mod.quarter_shape(H, W, D)
    out = torch.empty((Hq, Wq, 2), dtype=torch.float32, device="cuda")
    centre = torch.empty((H, W), dtype=torch.float32, device="cuda")
    conf = torch.empty((H, W), dtype=torch.float32, device="cuda")
    acts = torch.empty(_trace_sizes(Hq, Wq)[0], dtype=torch.float32, device="cuda")
    with fbs.Context(0) as ctx:
        fbs.fbs_band_net_set_params(ctx.ctx, theta)
        fbs.fbs_band_net_forward(ctx.ctx, _dev(L), _dev(R), H, W, 3, D, out, centre, conf)
        fbs.fbs_band_net_trace(ctx.ctx, acts, None)
        torch.cuda.synchronize()
        fbs.fbs_sync(ctx.ctx)
    (x0, ys, O), _ = br.split_trace(acts.cpu().numpy(), None, Hq, Wq)
    feat, est = _gpu_features(fbs, L, R, D)
    # the network input: the six features (checked against the FP64 oracle in
    # test_features_match_the_fp64_oracle) rounded to BF16, two zero channels
    assert np.array_equal(x0[..., :6], bn.round_bf16(feat)) and not x0[..., 6:].any()
    assert np.array_equal(O, out.cpu().numpy().astype(np.float64))
    th64 = theta.astype(np.float64)
    X = x0[..., :6]
    for l, (Wt, b) in enumerate(bn.unpack(th64)):
        Z, S = br.conv_with_scale(X, bn.round_bf16(Wt), b)
        eps = br.gamma(9 * bn.CIN[l] + 1) * S
        if l < bn.N_LAYERS - 1:
            defects, flips, amb = br.rounding_check(ys[l], Z, eps, relu=True)
            print(f"layer {l + 1}: {ys[l].size} activations, {amb} ambiguous, {flips} flips, {defects} defects")
            assert defects == 0, (l + 1, defects)
            X = ys[l]
        else:
            err = np.abs(O - Z)
            bound = eps + 2.0 ** -24 * np.abs(Z)
            print(f"outputs: max |err| / bound {float((err / bound).max()):.3f}")
            assert np.all(err <= bound)
    # end to end against the unrounded FP64 network (loose, reported)
    Of, _ = bn.forward(th64, feat.astype(np.float64))
    for c in range(2):
        e2e = np.linalg.norm(O[..., c] - Of[..., c]) / np.linalg.norm(Of[..., c])
        print(f"output {c}: rel. L2 vs the unrounded FP64 network {e2e:.2e}")
        assert e2e <= OUT_TOL, (c, e2e)
    # the head: centre = 4 (e* + o0) in FP32 and conf = sigmoid(z) of the
    # quarter pixel (x / 4, y / 4), from the kernel's own outputs
    g = out.cpu().numpy()
    up = bn.upsample(np.arange(Hq * Wq).reshape(Hq, Wq), H, W)
    o0 = g[..., 0].ravel()[up]
    z = g[..., 1].ravel()[up]
    expect_c = np.float32(4.0) * (est.ravel()[up].astype(np.float32) + o0)
    assert np.array_equal(centre.cpu().numpy(), expect_c)
    np.testing.assert_allclose(conf.cpu().numpy(), 1.0 / (1.0 + np.exp(-z.astype(np.float64))), rtol=0, atol=1e-6)


def test_backward_layers_match_elementwise(fbs, oracle_mod):
    from tests import _band_ref as br
    H, W, D, h = 120, 176, 64, 8
    L, R = _rand_pair(5, H, W, 3, shift=20)
    theta = _params(2)
    rng = np.random.default_rng(6)
    li = rng.integers(0, D, (H, W)).astype(np.int32)
    li[:, : W // 2] = 20                         # a region the band can cover
    ls = (li + rng.uniform(-0.5, 0.5, (H, W))).astype(np.float32)
    grad = np.zeros(bn.param_count(), np.float32)
    loss = np.zeros(1, np.float32)
    Hq, Wq, _ = oracle_mod.quarter_shape(H, W, D)
    na, ng = _trace_sizes(Hq, Wq)
    acts = torch.empty(na, dtype=torch.float32, device="cuda")
    grads = torch.empty(ng, dtype=torch.float32, device="cuda")
    with fbs.Context(0) as ctx:
        fbs.fbs_band_net_set_params(ctx.ctx, theta)
        fbs.fbs_band_net_train_step(ctx.ctx, _dev(L), _dev(R), H, W, 3, D, _dev(li), _dev(ls), h, 0.0, loss, grad)
        fbs.fbs_band_net_trace(ctx.ctx, acts, grads)
        torch.cuda.synchronize()
        fbs.fbs_sync(ctx.ctx)
    (x0, ys, O), (gs, go) = br.split_trace(acts.cpu().numpy(), grads.cpu().numpy(), Hq, Wq)
    feat, est = _gpu_features(fbs, L, R, D)
    th64 = theta.astype(np.float64)
    layers = bn.unpack(th64)
    N = Hq * Wq
    # loss and its gradient from the GPU's own outputs (targets from its centre)
    cq = 4.0 * (est + O[..., 0])
    t, y = oracle_mod.band_targets(li, ls, D, h, cq)
    Lref, dO = bn.loss_and_output_grad(O, est, t, y)
    assert abs(loss[0] - Lref) <= 1e-5 * abs(Lref) + 1e-7, (loss[0], Lref)
    eps_o = np.stack([2.0 ** -20 * 4.0 * np.abs(y) * (np.abs(cq) + np.abs(t) + 1.0),
                      2.0 ** -20 * (1.0 + np.abs(y))], axis=-1) / N
    defects, flips, amb = br.rounding_check(go[..., :2], dO, eps_o, relu=False)
    print(f"output gradient: {go[..., :2].size} values, {amb} ambiguous, {flips} flips, {defects} defects")
    assert defects == 0 and not go[..., 2:].any()
    inputs = [x0[..., :6]] + ys          # inputs[l] is the input of layer l + 1
    offs = np.cumsum([0] + [9 * ci * co + co for ci, co in zip(bn.CIN, bn.COUT)])
    G = go[..., :2]
    for l in range(bn.N_LAYERS - 1, -1, -1):
        ci, co = bn.CIN[l], bn.COUT[l]
        dW, db, dWa, dba = br.weight_grad_with_scale(inputs[l], G)
        gW = grad[offs[l]: offs[l] + 9 * ci * co].reshape(3, 3, ci, co).astype(np.float64)
        gb = grad[offs[l] + 9 * ci * co: offs[l + 1]].astype(np.float64)
        bW = br.gamma(N) * dWa + 2.0 ** -24 * np.abs(dW)
        bb = br.gamma(N) * dba + 2.0 ** -24 * np.abs(db)
        rW = float((np.abs(gW - dW) / np.maximum(bW, 1e-300)).max())
        print(f"layer {l + 1}: weight gradient max |err| / bound {rW:.3f}")
        assert np.all(np.abs(gW - dW) <= bW), l + 1
        assert np.all(np.abs(gb - db) <= bb), l + 1
        if l == 0:
            break
        dX, dXa = br.conv_transpose_with_scale(G, bn.round_bf16(layers[l][0]))
        mask = inputs[l] > 0
        eps = br.gamma(9 * co) * dXa
        defects, flips, amb = br.rounding_check(gs[l - 1], dX * mask, eps * mask, relu=False)
        print(f"layer {l}: {gs[l - 1].size} backward gradients, {amb} ambiguous, {flips} flips, {defects} defects")
        assert defects == 0, (l, defects)
        G = gs[l - 1]
    # end to end against the unrounded FP64 network (loose, reported)
    Of, actsf = bn.forward(th64, feat.astype(np.float64))
    cqf, _ = bn.centre_conf(Of, est)
    tf, yf = oracle_mod.band_targets(li, ls.astype(np.float64), D, h, cqf)
    Lf, dOf = bn.loss_and_output_grad(Of, est, tf, yf)
    gf = bn.backward(th64, actsf, dOf)
    assert abs(loss[0] - Lf) <= OUT_TOL * abs(Lf)
    for l, (ci, co) in enumerate(zip(bn.CIN, bn.COUT)):
        g = grad[offs[l]: offs[l + 1]]
        err = np.linalg.norm(g - gf[offs[l]: offs[l + 1]]) / np.linalg.norm(gf[offs[l]: offs[l + 1]])
        print(f"layer {l + 1}: rel. L2 vs the unrounded FP64 network {err:.2e}")
        assert err <= GRAD_TOL, (l, err)


def test_training_steps_reduce_the_loss(fbs, oracle_mod):
    """Labels 4 e* + 3 (a constant correction of the coarse winner that the
    network can represent through its biases): 100 Adam steps on one pair
    must cut the loss by more than half."""
    H, W, D = 160, 256, 128
    L, R = _rand_pair(21, H, W, 3, shift=24)
    _, est = _gpu_features(fbs, L, R, D)
    li = (4 * bn.upsample(est, H, W) + 3).astype(np.int32)
    ls = (li + 0.25).astype(np.float32)
    with fbs.Context(0) as ctx:
        dl, dr = _dev(L), _dev(R)
        fbs.fbs_band_net_init(ctx.ctx, 7)
        losses = []
        for it in range(100):
            loss = np.zeros(1, np.float32)
            fbs.fbs_band_net_train_step(ctx.ctx, dl, dr, H, W, 3, D, _dev(li), _dev(ls), 8, 1e-2, loss, None)
            losses.append(float(loss[0]))
    print("loss", losses[0], "->", losses[-1])
    assert np.all(np.isfinite(losses))
    assert np.mean(losses[-5:]) < 0.5 * np.mean(losses[:5]), losses


def test_params_round_trip_and_file(fbs, tmp_path):
    theta = _params(3)
    back = np.zeros_like(theta)
    with fbs.Context(0) as ctx:
        fbs.fbs_band_net_set_params(ctx.ctx, theta)
        fbs.fbs_band_net_get_params(ctx.ctx, back)
        assert np.array_equal(theta, back)
        path = str(tmp_path / "net.bin")
        fbs.fbs_band_net_save(ctx.ctx, path)
    with fbs.Context(0) as ctx:
        fbs.fbs_band_net_load(ctx.ctx, path)
        back2 = np.zeros_like(theta)
        fbs.fbs_band_net_get_params(ctx.ctx, back2)
        assert np.array_equal(theta, back2)
        fbs.fbs_band_net_init(ctx.ctx, 11)
        a = np.zeros_like(theta)
        fbs.fbs_band_net_get_params(ctx.ctx, a)
        fbs.fbs_band_net_init(ctx.ctx, 11)
        b = np.zeros_like(theta)
        fbs.fbs_band_net_get_params(ctx.ctx, b)
        assert np.array_equal(a, b) and np.all(np.isfinite(a)) and np.any(a != 0)


def test_learned_entry_equals_forward_then_banded(fbs):
    H, W, D = 120, 200, 64
    L, R = _rand_pair(12, H, W, 3, shift=14)
    with fbs.Context(0) as ctx:
        fbs.fbs_band_net_set_params(ctx.ctx, _params(4, 0.5))
        dl, dr = _dev(L), _dev(R)
        centre = torch.empty((H, W), dtype=torch.float32, device="cuda")
        conf = torch.empty((H, W), dtype=torch.float32, device="cuda")
        fbs.fbs_band_net_forward(ctx.ctx, dl, dr, H, W, 3, D, None, centre, conf)
        a = [torch.empty((H, W), dtype=torch.int32, device="cuda"), torch.empty((H, W), device="cuda")]
        b = [torch.empty((H, W), dtype=torch.int32, device="cuda"), torch.empty((H, W), device="cuda")]
        base = dict(left=dl, right=dr, H=H, W=W, C=3, D=D, radius=5, sigma_s=5.0, sigma_r=12.0, tau=0.0)
        fbs.fbs_compute_disparity_banded(ctx.ctx, dict(base, disp_int=a[0], disp_subpix=a[1]), centre, conf, 8, 0.5)
        fbs.fbs_compute_disparity_learned(ctx.ctx, dict(base, disp_int=b[0], disp_subpix=b[1]), 8, 0.5)
        torch.cuda.synchronize()
        fbs.fbs_sync(ctx.ctx)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_band_argument_validation(fbs):
    with fbs.Context(0) as ctx:
        x = torch.zeros((8, 8, 3), dtype=torch.uint8, device="cuda")
        o = torch.zeros((8, 8), dtype=torch.int32, device="cuda")
        c = torch.zeros((8, 8), device="cuda")
        pair = dict(left=x, right=x, H=8, W=8, C=3, D=16, radius=2, sigma_s=2.0, sigma_r=10.0, disp_int=o)
        with pytest.raises(fbs.FBSError):
            fbs.fbs_compute_disparity_banded(ctx.ctx, pair, c, c, 0, 0.5)
        with pytest.raises(fbs.FBSError):
            fbs.fbs_compute_disparity_banded(ctx.ctx, pair, None, c, 8, 0.5)
        with pytest.raises(fbs.FBSError):      # no weights yet
            fbs.fbs_compute_disparity_learned(ctx.ctx, pair, 8, 0.5)
        with pytest.raises(fbs.FBSError):
            fbs.fbs_band_net_set_params(ctx.ctx, np.zeros(5, np.float32))


@pytest.mark.parametrize("H,W,D,shift,th", [(37, 45, 40, 9, 0.05), (64, 200, 128, 24, 0.1), (23, 61, 16, 3, 0.0)])
def test_feature_points_match_the_oracle(fbs, oracle_mod, H, W, D, shift, th):
    L, R = _rand_pair(H + W + shift, H, W, 3, shift=shift)
    c = torch.empty((H, W), device="cuda")
    k = torch.empty((H, W), device="cuda")
    with fbs.Context(0) as ctx:
        fbs.fbs_band_feature_points(ctx.ctx, _dev(L), _dev(R), H, W, 3, D, th, c, k)
        torch.cuda.synchronize()
        fbs.fbs_sync(ctx.ctx)
    # exact wherever no margin in the pixel's window is within the FP32 bound of
    # theta and no winner there is within it of a tie
    rc, rk, amb = oracle_mod.band_feature_points(L, R, D, th, tol=2 * TOL_KBAR + 2 * U32)
    ok = ~amb
    print(f"{W}x{H} D={D} theta {th}: {int(amb.sum())} of {amb.size} pixels next to an undecided quarter pixel")
    assert ok.mean() >= 0.9
    assert np.array_equal(k.cpu().numpy()[ok], rk[ok])
    assert np.array_equal(c.cpu().numpy()[ok], rc[ok])
