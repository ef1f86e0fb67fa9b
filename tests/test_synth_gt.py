"""Ground truth, occlusion masks and evaluation regions of the synthetic
scenes, on scenes whose answers have closed forms (Table 1's regions and the
e_PEP of Eq. (11)-(12) rest on them)."""

import numpy as np

import oracle
from synth import Pair, regions, render_layers, shifted_texture_pair


def test_fronto_parallel_plane_over_background():
    """A fronto-parallel plane of disparity 11 over a background of disparity
    3: the ground truth is the plane's or the background's constant, and the
    background is hidden in the right view in a band of width 11 - 3 = 8 left
    of the plane (rows of the plane only) and where x - 3 leaves the image."""
    H, W, db, df = 64, 128, 3, 11
    x0, x1, y0, y1 = 40, 90, 10, 50
    left, right, gt, occ = render_layers(
        [("const", {"c": db}, "all"), ("const", {"c": df}, ("rect", x0, x1, y0, y1))], H, W, 3, seed=1)
    yy, xx = np.mgrid[0:H, 0:W]
    plane = (xx >= x0) & (xx < x1) & (yy >= y0) & (yy < y1)
    assert np.array_equal(gt, np.where(plane, float(df), float(db)))
    band = (yy >= y0) & (yy < y1) & (xx >= x0 - (df - db)) & (xx < x0)
    assert np.array_equal(occ, band | (~plane & (xx < db)))
    # every visible pixel appears at x - d in the right image (integer
    # disparities, no noise: the same texture sample)
    vis = ~occ
    ys, xs = np.nonzero(vis)
    assert np.array_equal(right[ys, xs - gt[ys, xs].astype(int)], left[ys, xs])


def test_slanted_plane_ground_truth_and_border():
    """One slanted plane d = a x + b y + c filling the image: the ground truth
    is the plane, and the only occlusion is where x - d(x, y) leaves the right
    image (x - d < -1/2)."""
    H, W = 48, 96
    a, b, c = 0.05, 0.02, 4.0
    _, _, gt, occ = render_layers([("plane", {"a": a, "b": b, "c": c}, "all")], H, W, 3, seed=2)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    expect = a * xx + b * yy + c
    np.testing.assert_allclose(gt, expect, rtol=0, atol=1e-12)
    assert np.array_equal(occ, xx - expect < -0.5)


def test_quadratic_surface_ground_truth():
    """A quadratic surface over the whole image: the ground truth is its
    closed form at every pixel."""
    H, W = 40, 80
    q = {"c": 6.0, "alpha": 0.002, "beta": 0.003, "x0": 30.0, "y0": 20.0}
    _, _, gt, _ = render_layers([("quad", q, "all")], H, W, 1, seed=3)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    np.testing.assert_allclose(gt, 6.0 + 0.002 * (xx - 30.0) ** 2 + 0.003 * (yy - 20.0) ** 2, rtol=0, atol=1e-12)


def test_shifted_texture_pair():
    """The known-answer pair: the left pixel x appears at x - d0 on the right."""
    L, R = shifted_texture_pair(20, 50, 3, 7, seed=4)
    assert np.array_equal(R[:, :50 - 7], L[:, 7:])


def test_regions_of_a_hand_built_scene():
    """Textured left half, flat right half; ground truth 5 left of column 30
    and 20 from it; a hand-drawn occlusion rectangle."""
    H, W = 40, 80
    rng = np.random.default_rng(5)
    left = np.full((H, W, 3), 128, np.uint8)
    left[:, : W // 2] = rng.integers(0, 256, size=(H, W // 2, 3))
    gt = np.where(np.arange(W)[None, :] < 30, 5.0, 20.0) * np.ones((H, 1))
    occ = np.zeros((H, W), bool)
    occ[5:10, 60:70] = True
    p = Pair(left=left, right=left.copy(), gt=gt, occ=occ, H=H, W=W, C=3, D=32, radius=3, sigma_s=3.0,
             sigma_r=12.0, tau=30.0)
    r = regions(p)
    assert np.array_equal(r["non_occ"], ~occ)
    tex = r["non_occ_textl"]
    assert tex[:, : W // 2 - 5].all() and not tex[:, W // 2 + 5:].any()
    # the step between columns 29 and 30 and its 3-pixel margin: columns 26 .. 33
    cols = np.arange(W)
    near = (cols >= 26) & (cols <= 33)
    assert np.array_equal(r["non_occ_discont"], ~occ & ~near[None, :])


def test_bench_e_pep_is_the_oracle_e_pep():
    """The sweep's e_PEP (bench.py) against the oracle's, which the golden
    example of Eq. (11)-(12) pins."""
    import bench
    rng = np.random.default_rng(6)
    est = rng.uniform(0, 64, (30, 40))
    truth = est + rng.normal(0, 2.5, est.shape)
    mask = rng.random(est.shape) < 0.7
    for eps in (0.5, 1.0, 2.0):
        assert bench.e_pep(est, truth, eps, mask) == oracle.e_pep(est, truth, eps, mask)
