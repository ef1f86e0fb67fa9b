"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks one part of the oracle against a library routine, a closed
form, an invariant or a special case that reduces to a textbook result, so a
dropped term, a wrong sign, a wrong index or a swapped operand in the oracle
fails at least one of them.
"""

import json
import os

import numpy as np
import pytest
from scipy import ndimage
from scipy.signal import windows

from synth import shifted_texture_pair

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_img(rng, H, W, C, lo=0, hi=256):
    return rng.integers(lo, hi, size=(H, W, C)).astype(np.uint8)


# ---------------------------------------------------------------------------
# Matching cost, Eq. (1)-(3)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("C", [1, 3])
def test_ncc_equals_pearson_correlation_bruteforce_8x8(oracle_mod, C):
    """Eq. (1)-(3) is the Pearson correlation of the two 3x3 blocks.

    numpy.corrcoef computes that correlation by its own formula; blocks are
    taken with replicate clamping, and for RGB the intensity is the channel
    sum (its correlation equals that of the channel mean).
    """
    rng = np.random.default_rng(11 + C)
    H = W = 8
    L = _rand_img(rng, H, W, C)
    R = _rand_img(rng, H, W, C)
    gl = L.astype(np.float64).sum(axis=2)
    gr = R.astype(np.float64).sum(axis=2)
    worst = 0.0
    for v in range(H):
        for u in range(W):
            for d in range(0, u + 1):
                ys = np.clip(np.arange(v - 1, v + 2), 0, H - 1)
                xl = np.clip(np.arange(u - 1, u + 2), 0, W - 1)
                xr = np.clip(np.arange(u - d - 1, u - d + 2), 0, W - 1)
                bl = gl[np.ix_(ys, xl)].ravel()
                br = gr[np.ix_(ys, xr)].ravel()
                if np.ptp(bl) == 0 or np.ptp(br) == 0:
                    expect = 0.0
                else:
                    expect = np.corrcoef(bl / C, br / C)[0, 1]
                got = oracle_mod.ncc(L, R, u, v, d)
                worst = max(worst, abs(got - expect))
    assert worst <= 1e-12


def test_ncc_affine_invariance_gives_plus_and_minus_one(oracle_mod):
    """i_r = a i_l + b with a > 0 gives c = 1; a < 0 gives c = -1 (no uint8 clipping)."""
    rng = np.random.default_rng(3)
    L = _rand_img(rng, 10, 12, 1, 0, 121)
    R_pos = (2 * L.astype(np.int32) + 10).astype(np.uint8)
    R_neg = (255 - L.astype(np.int32)).astype(np.uint8)
    for v in range(10):
        for u in range(12):
            if np.ptp(L[max(v - 1, 0):v + 2, max(u - 1, 0):u + 2]) == 0:
                continue
            assert abs(oracle_mod.ncc(L, R_pos, u, v, 0) - 1.0) < 1e-12
            assert abs(oracle_mod.ncc(L, R_neg, u, v, 0) + 1.0) < 1e-12


def test_cost_boundaries_flat_and_nomatch(oracle_mod):
    rng = np.random.default_rng(5)
    L = _rand_img(rng, 6, 9, 3)
    R = _rand_img(rng, 6, 9, 3)
    cv = oracle_mod.cost_volume(L, R, 7, oracle_mod.COST_NCC)
    # u - d < 0: no match, maximum cost 2
    for u in range(9):
        for d in range(7):
            if u - d < 0:
                assert cv[:, u, d].tolist() == [2.0] * 6
    assert cv.min() >= -1e-12 and cv.max() <= 2.0 + 1e-12
    # flat blocks: c := 0, so cost 1
    flat = np.full((5, 7, 1), 77, np.uint8)
    cvf = oracle_mod.cost_volume(flat, flat, 3, oracle_mod.COST_NCC)
    for u in range(7):
        for d in range(3):
            expect = 2.0 if u - d < 0 else 1.0
            assert np.all(cvf[:, u, d] == expect)


@pytest.mark.parametrize("delta,tau", [(7, 30.0), (45, 30.0), (0, 5.0)])
def test_tad_closed_form(oracle_mod, delta, tau):
    """TAD on two constant images: C = min(delta, tau), and tau where u - d < 0."""
    L = np.full((4, 6, 3), 100 + delta, np.uint8)
    R = np.full((4, 6, 3), 100, np.uint8)
    cv = oracle_mod.cost_volume(L, R, 4, oracle_mod.COST_TAD, tau)
    for u in range(6):
        for d in range(4):
            expect = tau if u - d < 0 else min(float(delta), tau)
            assert np.all(cv[:, u, d] == expect)


# ---------------------------------------------------------------------------
# Aggregation, Eq. (6)-(8)
# ---------------------------------------------------------------------------
def _gauss_kernel(radius, sigma_s):
    # scipy's Gaussian window exp(-n^2 / (2 std^2)); with std = sigma_s / sqrt(2)
    # it is the spatial weight of Eq. (7)
    g = windows.gaussian(2 * radius + 1, std=sigma_s / np.sqrt(2.0), sym=True)
    return np.outer(g, g)


@pytest.mark.parametrize("radius,sigma_s", [(2, 1.5), (4, 4.0), (3, 7.0)])
def test_constant_guide_reduces_to_normalised_gaussian_filter(oracle_mod, radius, sigma_s):
    """Constant guide => omega_r = 1 and Eq. (6) is a clipped, normalised
    Gaussian filter of every slice (scipy correlate with zero padding,
    divided by the filtered indicator of the image)."""
    rng = np.random.default_rng(radius)
    H, W, D = 9, 11, 3
    cost = rng.random((H, W, D))
    guide = np.full((H, W, 3), 90, np.uint8)
    agg = oracle_mod.aggregate(cost, guide, radius, sigma_s, 10.0)
    K = _gauss_kernel(radius, sigma_s)
    den = ndimage.correlate(np.ones((H, W)), K, mode="constant", cval=0.0)
    for d in range(D):
        num = ndimage.correlate(cost[:, :, d], K, mode="constant", cval=0.0)
        np.testing.assert_allclose(agg[:, :, d], num / den, rtol=0, atol=1e-12)


def test_large_sigma_s_gives_box_filter(oracle_mod):
    rng = np.random.default_rng(8)
    H, W, D, r = 7, 10, 2, 2
    cost = rng.random((H, W, D))
    guide = np.full((H, W, 1), 5, np.uint8)
    agg = oracle_mod.aggregate(cost, guide, r, 1e9, 10.0)
    den = ndimage.uniform_filter(np.ones((H, W)), size=2 * r + 1, mode="constant")
    for d in range(D):
        num = ndimage.uniform_filter(cost[:, :, d], size=2 * r + 1, mode="constant")
        np.testing.assert_allclose(agg[:, :, d], num / den, rtol=0, atol=1e-12)


def test_radius_zero_is_identity_and_constant_slice_is_kept(oracle_mod):
    rng = np.random.default_rng(9)
    cost = rng.random((6, 7, 4))
    guide = _rand_img(rng, 6, 7, 3)
    assert np.array_equal(oracle_mod.aggregate(cost, guide, 0, 3.0, 10.0), cost)
    const = np.full((6, 7, 2), 0.625)
    np.testing.assert_allclose(oracle_mod.aggregate(const, guide, 3, 3.0, 10.0), const, atol=1e-14)


def test_range_weight_closed_form_on_two_level_guide(oracle_mod):
    """Two-colour guide, omega_d ~ 1 (huge sigma_s), cost 1 on region A and 0 on B.

    At a pixel of A whose window holds n_A pixels of A and n_B of B,
    Eq. (6)-(8) give n_A / (n_A + n_B exp(-|a - b|^2 / gamma_r^2)) with the
    squared Euclidean colour distance and no factor 2.
    """
    H, W, r, sr = 5, 8, 2, 20.0
    a = np.array([100, 120, 90])
    b = np.array([110, 100, 95])
    guide = np.empty((H, W, 3), np.uint8)
    guide[:, :4] = a
    guide[:, 4:] = b
    cost = np.zeros((H, W, 1))
    cost[:, :4, 0] = 1.0
    agg = oracle_mod.aggregate(cost, guide, r, 1e9, sr)
    e = np.exp(-float(np.sum((a - b) ** 2)) / sr ** 2)
    # pixel (u=3, v=2): window x 1..5, y 0..4 -> A columns 1..3 (3), B columns 4..5 (2)
    nA, nB = 3 * 5, 2 * 5
    assert abs(agg[2, 3, 0] - nA / (nA + nB * e)) < 1e-12
    # pixel (u=0, v=0): window x 0..2, y 0..2 (clipped) -> all A
    assert abs(agg[0, 0, 0] - 1.0) < 1e-12
    # pixel (u=4, v=4): window x 2..6, y 2..4 -> A columns 2..3 (2), B 4..6 (3), 3 rows
    nA, nB = 2 * 3, 3 * 3
    assert abs(agg[4, 4, 0] - nA * e / (nA * e + nB)) < 1e-12


def test_aggregation_is_linear_in_cost_and_flip_equivariant(oracle_mod):
    rng = np.random.default_rng(12)
    H, W, D = 7, 9, 3
    guide = _rand_img(rng, H, W, 3)
    c1, c2 = rng.random((H, W, D)), rng.random((H, W, D))
    f = lambda c, g=guide: oracle_mod.aggregate(c, g, 2, 2.5, 15.0)
    np.testing.assert_allclose(f(0.3 * c1 - 1.7 * c2), 0.3 * f(c1) - 1.7 * f(c2), atol=1e-12)
    flipped = f(c1[:, ::-1].copy(), guide[:, ::-1].copy())
    np.testing.assert_allclose(flipped[:, ::-1], f(c1), atol=1e-13)
    flipped_v = f(c1[::-1].copy(), guide[::-1].copy())
    np.testing.assert_allclose(flipped_v[::-1], f(c1), atol=1e-13)


def test_aggregation_matches_dense_matrix_form_8x8(oracle_mod):
    """Brute force on 8x8: Agg = (Wm @ C) / Wm.sum(1) with Wm built from
    pairwise distance arrays (a different route through the same definition)."""
    rng = np.random.default_rng(21)
    H = W = 8
    r, ss, sr = 3, 2.0, 25.0
    guide = _rand_img(rng, H, W, 3)
    cost = rng.random((H, W, 5))
    yy, xx = np.mgrid[0:H, 0:W]
    P = np.stack([xx.ravel(), yy.ravel()], 1).astype(np.float64)
    G = guide.reshape(-1, 3).astype(np.float64)
    dxy = P[:, None, :] - P[None, :, :]
    inwin = (np.abs(dxy) <= r).all(axis=2)
    Wm = np.exp(-(dxy ** 2).sum(2) / ss ** 2) * np.exp(-((G[:, None] - G[None]) ** 2).sum(2) / sr ** 2)
    Wm *= inwin
    expect = (Wm @ cost.reshape(-1, 5)) / Wm.sum(1, keepdims=True)
    got = oracle_mod.aggregate(cost, guide, r, ss, sr).reshape(-1, 5)
    np.testing.assert_allclose(got, expect, atol=1e-12)


# ---------------------------------------------------------------------------
# WTA and subpixel, Eq. (10)
# ---------------------------------------------------------------------------
def test_wta_matches_numpy_argmin_first_occurrence(oracle_mod):
    rng = np.random.default_rng(4)
    agg = rng.integers(0, 5, size=(40, 9)).astype(np.float64)   # many exact ties
    di, _ = oracle_mod.wta_subpixel(agg)
    assert np.array_equal(di, np.argmin(agg, axis=1))


def test_subpixel_returns_vertex_of_exact_quadratic(oracle_mod):
    D = 16
    d = np.arange(D, dtype=np.float64)
    for dv in [3.0, 3.25, 7.49, 7.5, 10.8, 1.0 - 0.4999]:
        for alpha, beta in [(0.01, 0.3), (2.0, -1.0), (1e-3, 0.5)]:
            agg = alpha * (d - dv) ** 2 + beta
            di, ds = oracle_mod.wta_subpixel(agg[None])
            assert di[0] == int(np.floor(dv + 0.5)) or abs(dv - np.floor(dv) - 0.5) < 1e-9
            assert abs(ds[0] - dv) < 1e-9


def test_subpixel_agrees_with_polyfit_and_stays_in_half_pixel(oracle_mod):
    rng = np.random.default_rng(6)
    agg = rng.random((300, 12))
    di, ds = oracle_mod.wta_subpixel(agg)
    for p in range(300):
        b = di[p]
        off = ds[p] - b
        assert -0.5 < off <= 0.5
        if 0 < b < 11:
            c2, c1, _ = np.polyfit([-1.0, 0.0, 1.0], agg[p, b - 1:b + 2], 2)
            assert abs(off - (-c1 / (2 * c2))) < 1e-9
        else:
            assert off == 0.0


# ---------------------------------------------------------------------------
# End to end
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("C,d0,r", [(1, 5, 2), (3, 9, 3)])
def test_shifted_texture_recovers_disparity_exactly(oracle_mod, C, d0, r):
    """Right = left shifted by d0 (noise-free): cost 0 at d0 wherever both
    blocks are unclamped, hence aggregated cost 0 and d* = d0 in the interior."""
    H, W, D = 16, 40, 14
    L, R = shifted_texture_pair(H, W, C, d0, seed=7 + C)
    di, ds, agg = oracle_mod.fbs(L, R, D, r, float(r), 12.0, want_agg=True)
    x0, x1 = d0 + 1 + r, W - 2 - r
    assert x1 > x0
    interior = np.s_[:, x0:x1 + 1]
    assert np.all(np.abs(agg[interior][..., d0]) < 1e-12)
    assert np.all(di[interior] == d0)
    assert np.all(np.abs(ds[interior] - d0) <= 0.5)


def test_points_and_rows_agree(oracle_mod):
    """The pointwise evaluation and the row-band evaluation are two routes
    through the oracle; they must agree to rounding."""
    rng = np.random.default_rng(2)
    L = _rand_img(rng, 12, 20, 3)
    R = _rand_img(rng, 12, 20, 3)
    di, ds, agg = oracle_mod.fbs(L, R, 8, 2, 2.0, 12.0, want_agg=True)
    xs = np.array([0, 5, 19, 11])
    ys = np.array([0, 6, 11, 3])
    pi, ps, pagg = oracle_mod.fbs_points(L, R, 8, 2, 2.0, 12.0, xs, ys)
    np.testing.assert_allclose(pagg, agg[ys, xs], atol=1e-13)
    assert np.array_equal(pi, di[ys, xs])
    band_i, band_s, band_agg = oracle_mod.fbs(L, R, 8, 2, 2.0, 12.0, rows=(4, 9), want_agg=True)
    np.testing.assert_allclose(band_agg, agg[4:9], atol=1e-13)


def test_e_pep_golden(oracle_mod):
    with open(os.path.join(GOLDEN, "e_pep_example.json")) as f:
        g = json.load(f)
    est = np.array(g["estimate"])
    gt = np.array(g["truth"])
    assert oracle_mod.e_pep(est, gt, g["eps"]) == pytest.approx(g["expected_percent"])
    mask = np.array(g["mask"], bool)
    assert oracle_mod.e_pep(est, gt, g["eps"], mask) == pytest.approx(g["expected_percent_masked"])


def test_mde_per_s_formula(oracle_mod):
    # Eq. (13): u_max v_max d_max / t * 1e-6
    assert oracle_mod.mde_per_s(450, 375, 60, 0.5) == pytest.approx(20.25)


# ---------------------------------------------------------------------------
# Right view and the left-right consistency check, Eq. (9)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mode,C", [(0, 3), (1, 1)])
def test_right_view_is_the_mirrored_left_view_of_the_swapped_pair(oracle_mod, mode, C):
    """Mirroring both images and swapping them turns the right view into a
    left view: right_fbs(L, R) = mirror(left_fbs(mirror(R), mirror(L))).  This
    goes through the pinned left path by an independent route."""
    rng = np.random.default_rng(31 + mode)
    H, W, D, r = 9, 23, 7, 2
    L = _rand_img(rng, H, W, C)
    R = np.roll(L, -2, axis=1)
    R[:, -2:] = _rand_img(rng, H, 2, C)
    di, ds, agg = oracle_mod.fbs_right(L, R, D, r, 2.0, 10.0, tau=25.0, mode=mode, want_agg=True)
    mi, ms, magg = oracle_mod.fbs(R[:, ::-1], L[:, ::-1], D, r, 2.0, 10.0, tau=25.0, mode=mode, want_agg=True)
    np.testing.assert_allclose(agg, magg[:, ::-1], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(di, mi[:, ::-1])
    np.testing.assert_allclose(ds, ms[:, ::-1], rtol=0, atol=1e-9)


def test_lrc_on_a_shifted_texture(oracle_mod):
    """Right = left shifted by d0 (noise free): every left pixel with a match
    (x >= d0) away from the borders is confirmed, and the unmatched strip
    x < d0 - 1 is rejected wherever its left winner is not the true d0."""
    H, W, D, d0, r = 12, 40, 12, 5, 2
    L, R = shifted_texture_pair(H, W, 1, d0, seed=4)
    dl, _ = oracle_mod.fbs(L, R, D, r, 2.0, 10.0)
    dr, _ = oracle_mod.fbs_right(L, R, D, r, 2.0, 10.0)
    ok = oracle_mod.lrc(dl, dr)
    assert np.all(dl[r + 1:-r - 1, d0 + r + 1:-r - 1] == d0)
    assert np.all(dr[r + 1:-r - 1, r + 1:W - d0 - r - 1] == d0)
    assert np.all(ok[r + 1:-r - 1, d0 + r + 1:-r - 1] == 1)
    strip = ok[:, :d0]
    assert np.all(strip[dl[:, :d0] > np.arange(d0)[None, :]] == 0)   # u - d < 0 is never confirmed


def test_lrc_definition_bruteforce(oracle_mod):
    rng = np.random.default_rng(2)
    dl = rng.integers(0, 6, (5, 9)).astype(np.int32)
    dr = rng.integers(0, 6, (5, 9)).astype(np.int32)
    ok = oracle_mod.lrc(dl, dr)
    for v in range(5):
        for u in range(9):
            d = dl[v, u]
            assert ok[v, u] == int(u - d >= 0 and dr[v, u - d] == d)
