"""Pins of the band form's oracle (band_oracle.c, band_net.py).

Each check compares the oracle with a library routine, a closed form, finite
differences or a brute-force restatement, so that a dropped term, a wrong
sign, a transposed operand or an off-by-one in a band edge fails one of them.
"""

import numpy as np
import pytest
from scipy import signal

from oracle import band_net as bn
from synth import shifted_texture_pair


# ---------------------------------------------------------------------------
# Quarter-resolution features (readings B1-B3)
# ---------------------------------------------------------------------------
def test_downsample_constant_and_clamped_edges(oracle_mod):
    img = np.full((6, 7, 3), 9, np.uint8)
    assert np.all(oracle_mod.band_downsample(img) == 16 * 3 * 9)
    # a single bright pixel in the last column: every block that clamps onto
    # that column counts it once per clamped sample
    g = np.zeros((4, 5, 1), np.uint8)
    g[0, 4, 0] = 1
    q = oracle_mod.band_downsample(g)
    assert q.shape == (1, 2)
    assert q[0, 0] == 0 and q[0, 1] == 4     # x = 4,5,6,7 all clamp to column 4


def test_coarse_cost_matches_pearson_in_fp64(oracle_mod):
    """The coarse cost is 1 - corrcoef of the two clamped 3x3 blocks of quarter
    intensities (numpy's own formula), averaged over the 5x5 quarter window
    clipped to the image: f2 at the winner matches it to FP64 accuracy, the
    winner is its argmin (except at ties closer than the FP64 rounding of two
    different formulas), f3..f5 follow, and the reported gap is the distance
    from the best to the second best."""
    rng = np.random.default_rng(3)
    H, W, D = 24, 40, 24
    L = rng.integers(0, 256, size=(H, W, 3)).astype(np.uint8)
    R = rng.integers(0, 256, size=(H, W, 3)).astype(np.uint8)
    feat, est, gap = oracle_mod.band_features(L, R, D, with_gap=True)
    gl = oracle_mod.band_downsample(L).astype(np.float64)
    gr = oracle_mod.band_downsample(R).astype(np.float64)
    Hq, Wq, Dq = oracle_mod.quarter_shape(H, W, D)
    K = np.full((Hq, Wq, Dq), 2.0)
    for Y in range(Hq):
        ys = np.clip(np.arange(Y - 1, Y + 2), 0, Hq - 1)
        for X in range(Wq):
            for e in range(X + 1 if X + 1 < Dq else Dq):
                bl = gl[np.ix_(ys, np.clip(np.arange(X - 1, X + 2), 0, Wq - 1))].ravel()
                br = gr[np.ix_(ys, np.clip(np.arange(X - e - 1, X - e + 2), 0, Wq - 1))].ravel()
                K[Y, X, e] = 1.0 if (np.ptp(bl) == 0 or np.ptp(br) == 0) else 1.0 - np.corrcoef(bl, br)[0, 1]
    for Y in range(Hq):
        for X in range(Wq):
            win = K[max(0, Y - 2):Y + 3, max(0, X - 2):X + 3]
            Kb = win.reshape(-1, Dq).mean(axis=0)
            e = est[Y, X]
            assert abs(feat[Y, X, 2] - Kb[e]) <= 1e-12
            srt = np.sort(Kb)
            if srt[1] - srt[0] > 1e-12:
                assert e == np.argmin(Kb)
            assert abs(gap[Y, X] - (srt[1] - srt[0])) <= 1e-12
            assert feat[Y, X, 1] == e / Dq
            k2 = min([Kb[j] for j in range(Dq) if abs(j - e) >= 2] + [2.0])
            assert abs(feat[Y, X, 3] - min(k2 - Kb[e], 1.0)) <= 1e-12
            km = Kb[e - 1] if e > 0 else 2.0
            kp = Kb[e + 1] if e < Dq - 1 else 2.0
            assert abs(feat[Y, X, 4] - (km - Kb[e])) <= 1e-12
            assert abs(feat[Y, X, 5] - (kp - Kb[e])) <= 1e-12
            assert abs(feat[Y, X, 0] - (gl[Y, X] / (16 * 255 * 3) - 0.5)) <= 1e-15


@pytest.mark.parametrize("k", [2, 5])
def test_coarse_winner_recovers_a_shift_by_four_k(oracle_mod, k):
    """Right = left shifted by 4k pixels: the quarter planes are shifted by
    exactly k, so away from the borders (block clamping and the 5x5 window)
    the coarse winner is k with cost ~0."""
    H, W, D = 48, 96, 64
    L, R = shifted_texture_pair(H, W, 3, 4 * k, seed=k)
    feat, est = oracle_mod.band_features(L, R, D)
    interior = est[3:-3, k + 3:-3]
    assert np.all(interior == k)
    assert np.all(np.abs(feat[3:-3, k + 3:-3, 2]) <= 1e-12)


# ---------------------------------------------------------------------------
# Band limits (B4) and band FBS (B5)
# ---------------------------------------------------------------------------
def test_band_limits_closed_cases(oracle_mod):
    D, h, th = 64, 8, 0.5
    c = np.array([10.49, 10.5, -3.0, 70.0, np.nan, 30.0, 30.0, 3.2], np.float32)
    k = np.array([0.9, 0.9, 0.9, 0.9, 0.9, 0.2, np.nan, 0.5], np.float32)
    lo, hi = oracle_mod.band_limits(c, k, D, h, th)
    assert lo.tolist() == [2, 3, 0, 55, 0, 0, 0, 0]
    assert hi.tolist() == [18, 19, 8, 63, 63, 63, 63, 11]


def test_band_fbs_full_range_equals_plain_fbs(oracle_mod):
    rng = np.random.default_rng(5)
    H, W, D, r = 10, 14, 12, 2
    L = rng.integers(0, 256, size=(H, W, 3)).astype(np.uint8)
    R = np.roll(L, -2, axis=1)
    ys, xs = np.mgrid[0:H, 0:W]
    xs, ys = xs.ravel(), ys.ravel()
    n = xs.size
    di, ds, agg = oracle_mod.fbs_band_points(L, R, D, r, 2.0, 12.0, xs, ys, np.zeros(n), np.full(n, D - 1))
    rdi, rds, ragg = oracle_mod.fbs_points(L, R, D, r, 2.0, 12.0, xs, ys)
    assert np.array_equal(di, rdi)
    assert np.array_equal(ds, rds)
    assert np.array_equal(agg, ragg)


def test_band_fbs_bruteforce_8x8(oracle_mod):
    """Brute force: restrict the plain aggregated volume to each band, take
    the first minimum, and apply Eq. (10) only inside the band."""
    rng = np.random.default_rng(8)
    H = W = 8
    D, r = 8, 2
    L = rng.integers(0, 256, size=(H, W, 1)).astype(np.uint8)
    R = rng.integers(0, 256, size=(H, W, 1)).astype(np.uint8)
    agg = oracle_mod.aggregate(oracle_mod.cost_volume(L, R, D), L, r, 2.0, 10.0)
    ys, xs = np.mgrid[0:H, 0:W]
    xs, ys = xs.ravel(), ys.ravel()
    lo = rng.integers(0, D, xs.size)
    hi = np.minimum(lo + rng.integers(0, 4, xs.size), D - 1)
    di, ds, bagg = oracle_mod.fbs_band_points(L, R, D, r, 2.0, 10.0, xs, ys, lo, hi)
    for i in range(xs.size):
        a = agg[ys[i], xs[i]]
        b0, b1 = lo[i], hi[i]
        best = b0
        for d in range(b0 + 1, b1 + 1):
            if a[d] < a[best]:
                best = d
        assert di[i] == best
        expect = float(best)
        if b0 < best < b1:
            den = 2 * a[best - 1] + 2 * a[best + 1] - 4 * a[best]
            if den > 0:
                expect = best + (a[best - 1] - a[best + 1]) / den
        assert abs(ds[i] - expect) <= 1e-12
        np.testing.assert_allclose(bagg[i, b0:b1 + 1], a[b0:b1 + 1], rtol=0, atol=1e-12)
        assert np.all(np.isnan(bagg[i, :b0])) and np.all(np.isnan(bagg[i, b1 + 1:]))


def test_band_targets_small_case(oracle_mod):
    H, W, D, h = 5, 6, 32, 4
    li = np.full((H, W), 10, np.int32)
    ls = np.full((H, W), 10.25, np.float32)
    li[0, 0], ls[0, 0] = 200, 200.5      # one outlier in quarter pixel (0, 0)
    li[4, 5], ls[4, 5] = 14, 14.25       # quarter pixel (1, 1) holds only pixels (4, 4) and (4, 5)
    li[1, 4], ls[1, 4] = 11, 11.0        # quarter pixel (0, 1) holds 8 pixels: 7 x 10.25, 1 x 11.0
    cq = np.array([[10.0, 10.6], [13.4, 10.4]])
    t, y = oracle_mod.band_targets(li, ls, D, h, cq)
    assert t[0, 0] == 10.25              # the median ignores the outlier
    assert t[0, 1] == 10.25              # even count: mean of the two middle values (10.25, 10.25)
    assert t[1, 0] == 10.25
    assert t[1, 1] == (10.25 + 14.25) / 2
    # bands [m-3, m+3]: m = 10 -> [7, 13]; m = 11 -> [8, 14]; m = 13 -> [10, 16]; m = 10 -> [7, 13]
    assert y[0, 0] == 15 / 16 and y[0, 1] == 1.0 and y[1, 0] == 1.0 and y[1, 1] == 0.5


# ---------------------------------------------------------------------------
# Network (band_net.py)
# ---------------------------------------------------------------------------
def test_conv3x3_matches_scipy_correlate():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((7, 9, 3))
    Wt = rng.standard_normal((3, 3, 3, 4))
    b = rng.standard_normal(4)
    out = bn.conv3x3(X, Wt, b)
    for o in range(4):
        ref = b[o] + sum(signal.correlate2d(X[:, :, i], Wt[:, :, i, o], mode="same", boundary="fill")
                         for i in range(3))
        np.testing.assert_allclose(out[:, :, o], ref, rtol=0, atol=1e-12)


def _small_problem(seed=0, Hq=6, Wq=7):
    rng = np.random.default_rng(seed)
    theta = rng.standard_normal(bn.param_count()) * 0.15
    feat = rng.standard_normal((Hq, Wq, bn.N_FEATURES))
    est = rng.integers(0, 16, (Hq, Wq))
    t = rng.uniform(0, 64, (Hq, Wq))
    y = rng.integers(0, 2, (Hq, Wq))
    return theta, feat, est, t, y


def _loss(theta, feat, est, t, y):
    O, _ = bn.forward(theta, feat)
    return bn.loss_and_output_grad(O, est, t, y)[0]


def test_network_gradient_matches_central_differences():
    theta, feat, est, t, y = _small_problem()
    O, acts = bn.forward(theta, feat)
    _, dO = bn.loss_and_output_grad(O, est, t, y)
    g = bn.backward(theta, acts, dO)
    rng = np.random.default_rng(2)
    # a sample of coordinates from every layer's weights and biases
    idx, o = [], 0
    for ci, co in zip(bn.CIN, bn.COUT):
        idx += list(o + rng.choice(9 * ci * co, 6, replace=False))
        idx += list(o + 9 * ci * co + rng.choice(co, 2, replace=False))
        o += 9 * ci * co + co
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (_loss(theta + e, feat, est, t, y) - _loss(theta - e, feat, est, t, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_loss_closed_forms():
    O = np.zeros((1, 2, 2))
    est = np.array([[2, 3]])
    # c = 4 e*: errors 0 and 2 -> huber 0 and 1.5, weighted by y = 1 and 0.5;
    # z = 0 -> bce = log 2 for any y
    L, dO = bn.loss_and_output_grad(O, est, np.array([[8.0, 10.0]]), np.array([[1.0, 0.5]]))
    assert abs(L - (0.0 + 0.75 + 2 * np.log(2.0)) / 2) <= 1e-15
    assert np.allclose(dO[0, :, 0], [0.0, 4.0 * 0.5 * 1.0 / 2])
    assert np.allclose(dO[0, :, 1], [(0.5 - 1) / 2, 0.0])


def test_adam_first_step_closed_form():
    """After one step m_hat = g and v_hat = g^2, so each coordinate moves by
    lr * g / (|g| + eps)."""
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    th = np.array([1.0, 1.0, 1.0, 1.0])
    new, m, v = bn.adam_step(th, np.zeros(4), np.zeros(4), g, 1, 0.01)
    np.testing.assert_allclose(new, th - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_upsample_nearest():
    q = np.arange(6).reshape(2, 3)
    up = bn.upsample(q, 7, 10)
    assert up.shape == (7, 10)
    assert up[6, 9] == q[1, 2] and up[3, 3] == q[0, 0] and up[4, 4] == q[1, 1]


def test_round_bf16_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    x = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-8, 8, 10000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 3e38, -1e-38]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(bn.round_bf16(x), ref)


def test_bf16_mode_changes_only_operands():
    """With every operand already a BF16 value and biases / inputs chosen so
    that all activations stay BF16-exact (integers of small magnitude), the
    rounded network equals the plain one."""
    rng = np.random.default_rng(10)
    theta = np.zeros(bn.param_count())
    o = 0
    for ci, co in zip(bn.CIN, bn.COUT):
        n = 9 * ci * co
        theta[o:o + n] = rng.integers(-1, 2, n) * (rng.random(n) < 0.05)
        o += n + co
    feat = rng.integers(0, 3, (5, 6, bn.N_FEATURES)).astype(np.float64)
    O1, a1 = bn.forward(theta, feat)
    O2, a2 = bn.forward(theta, feat, bf16=True)
    if max(np.abs(a).max() for a in a1) >= 256:
        pytest.skip("activations left the exactly representable range")
    assert np.array_equal(O1, O2)
    dO = rng.integers(-2, 3, O1.shape).astype(np.float64)
    assert np.array_equal(bn.backward(theta, a1, dO), bn.backward(theta, a2, dO, bf16=True))


def test_feature_point_proposal_definition(oracle_mod):
    """B7 restated with numpy from the pinned features: the 5x5 quarter window
    of feature points (margin >= theta), their count and winner spread."""
    rng = np.random.default_rng(12)
    H, W, D, th = 30, 45, 32, 0.05
    L = rng.integers(0, 256, size=(H, W, 3)).astype(np.uint8)
    R = np.roll(L, -8, axis=1)
    feat, est, gap = oracle_mod.band_features(L, R, D, with_gap=True)
    tol = 1e-3
    c, k, amb = oracle_mod.band_feature_points(L, R, D, th, tol=tol)
    assert np.array_equal(oracle_mod.band_feature_points(L, R, D, th), (c, k))
    Hq, Wq = est.shape
    fp = feat[..., 3] >= th
    undecided = (np.abs(feat[..., 3] - th) <= tol) | (gap <= tol)
    for y in range(H):
        for x in range(W):
            Y, X = y // 4, x // 4
            win = (slice(max(0, Y - 2), Y + 3), slice(max(0, X - 2), X + 3))
            e = est[win][fp[win]]
            if e.size >= 3 and e.max() - e.min() <= 2:
                assert k[y, x] == 1.0 and c[y, x] == 2.0 * (e.max() + e.min())
            else:
                assert k[y, x] == 0.0
            assert amb[y, x] == undecided[win].any()


def test_feature_points_on_a_shift_by_four_k(oracle_mod):
    """Shift by 4k: away from the borders every pixel is confident with centre 4k."""
    H, W, D, k = 64, 128, 64, 6
    L, R = shifted_texture_pair(H, W, 3, 4 * k, seed=2)
    c, conf = oracle_mod.band_feature_points(L, R, D, 0.05)
    inner = (slice(20, -20), slice(4 * k + 24, -20))
    assert np.all(conf[inner] == 1.0) and np.all(c[inner] == 4.0 * k)


def test_layer_check_helper_separates_flips_from_defects():
    """The element-wise rule of tests/_band_ref.py: the BF16 rounding of the
    FP64 value passes; the other rounding passes only where the value lies
    within the accumulation bound of a rounding midpoint (a flip); any other
    value is a defect."""
    from tests import _band_ref as br
    one_ulp = 2.0 ** -7                        # BF16 spacing in [1, 2)
    mid = 1.0 + 0.5 * one_ulp                  # midpoint between 1 and 1 + ulp
    z = np.array([1.3, mid - 1e-6, mid + 1e-6, mid - 1e-3, 2.0 ** -30, -1e-12])
    eps = np.full(z.shape, 1e-5)
    exact = bn.round_bf16(np.maximum(z, 0.0))
    assert br.rounding_check(exact, z, eps, relu=True)[0] == 0
    # the other rounding next to the midpoint: a flip, not a defect
    got = exact.copy()
    got[1] = 1.0 + one_ulp
    got[2] = 1.0
    d, f, a = br.rounding_check(got, z, eps, relu=True)
    assert (d, f) == (0, 2) and a >= 2
    # the other rounding far from the midpoint: a defect
    got = exact.copy()
    got[3] = 1.0 + one_ulp
    assert br.rounding_check(got, z, eps, relu=True)[0] == 1
    # a wrong value (a mis-indexed tap would give one): a defect
    got = exact.copy()
    got[0] = bn.round_bf16(np.array([1.5]))[0]
    assert br.rounding_check(got, z, eps, relu=True)[0] == 1
    # at the ReLU boundary both 0 and a small positive value pass
    got = exact.copy()
    got[4] = 0.0
    got[5] = bn.round_bf16(np.array([1e-12]))[0]
    assert br.rounding_check(got, z, np.full(z.shape, 1e-9), relu=True)[0] == 0
    # signed values without ReLU
    s = np.array([-1.3, -(mid - 1e-6)])
    e2 = np.full(2, 1e-5)
    assert br.rounding_check(bn.round_bf16(s), s, e2, relu=False)[0] == 0
    assert br.rounding_check(np.array([bn.round_bf16(np.array([-1.3]))[0], -(1.0 + one_ulp)]), s, e2,
                             relu=False)[:2] == (0, 1)
    assert br.rounding_check(np.array([1.3, -1.0]), s, e2, relu=False)[0] == 1
