"""What the trained band network gains over the band path without it.

On held-out 1920x1080 RGB pairs (D = 256, radius 9; scene seeds outside the
training and validation sets) three results are compared with the plain
full-range FP32 path, pixel by pixel (> 1 px counts as bad):

  * learned: the shipped network's centres and confidences (the threshold
             recorded with the weights);
  * coarse:  the same band rule around the coarse winner alone, c = 4 e*,
             falling back to the full range on the same fraction of pixels,
             chosen by the coarse cost margin (feature f3): the method
             without the network at equal work;
  * the learned result must stay within 0.5% extra bad pixels of the plain
    path while leaving at most half of the full-range aggregation work, and
    stay below the coarse result's bad-pixel rate.
"""

import os

import numpy as np
import pytest

from oracle import band_net as bn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WORKLOAD = "rgb1920x1080_d256_r9"
HALF_BAND = 8


@pytest.fixture(scope="module")
def fbs():
    from paper_1807_02044_gb300 import build as b
    b.build()
    import paper_1807_02044_gb300 as m
    return m


def _banded(fbs, ctx, dl, dr, p, centre, conf, threshold):
    di = torch.empty((p.H, p.W), dtype=torch.int32, device="cuda")
    ds = torch.empty((p.H, p.W), device="cuda")
    fbs.fbs_compute_disparity_banded(ctx.ctx, dict(left=dl, right=dr, H=p.H, W=p.W, C=3, D=p.D, radius=p.radius,
                                                   sigma_s=p.sigma_s, sigma_r=p.sigma_r, disp_int=di,
                                                   disp_subpix=ds), centre, conf, HALF_BAND, threshold)
    return ds


@pytest.mark.parametrize("seed", [11, 12])
def test_trained_network_beats_the_coarse_band_at_equal_work(fbs, oracle_mod, seed):
    from synth import make_pair
    path = fbs.default_band_net_path()
    assert os.path.exists(path), "the trained weights ship with the package"
    p = make_pair(WORKLOAD, seed)
    H, W, D = p.H, p.W, p.D
    thr = fbs.default_band_threshold()
    with fbs.Context(0) as ctx:
        fbs.fbs_band_net_load(ctx.ctx, path)
        dl = torch.from_numpy(p.left).cuda()
        dr = torch.from_numpy(p.right).cuda()
        _, plain = ctx.compute_disparity(dl, dr, D, p.radius, p.sigma_s, p.sigma_r)
        centre = torch.empty((H, W), device="cuda")
        conf = torch.empty((H, W), device="cuda")
        fbs.fbs_band_net_forward(ctx.ctx, dl, dr, H, W, 3, D, None, centre, conf)
        learned = _banded(fbs, ctx, dl, dr, p, centre, conf, thr)
        fallback = float((conf < thr).float().mean().item())
        lo = torch.empty((H, W), dtype=torch.int32, device="cuda")
        hi = torch.empty((H, W), dtype=torch.int32, device="cuda")
        fbs.fbs_band_limits(ctx.ctx, centre, conf, H * W, D, HALF_BAND, thr, lo, hi)
        torch.cuda.synchronize()
        work = float(((hi - lo + 1).double().sum() / (H * W * D)).item())
        # the coarse band: centre 4 e*, the same fallback fraction by lowest margin
        Hq, Wq, _ = oracle_mod.quarter_shape(H, W, D)
        feat = torch.empty((Hq, Wq, 6), device="cuda")
        est = torch.empty((Hq, Wq), dtype=torch.int32, device="cuda")
        fbs.fbs_band_features(ctx.ctx, dl, dr, H, W, 3, D, feat, est)
        torch.cuda.synchronize()
        up = bn.upsample(np.arange(Hq * Wq).reshape(Hq, Wq), H, W)
        c0 = (4.0 * est.cpu().numpy().ravel()[up]).astype(np.float32)
        margin = feat[..., 3].cpu().numpy().ravel()[up]
        cut = np.quantile(margin, fallback) if fallback > 0 else -np.inf
        k0 = (margin >= cut).astype(np.float32)
        coarse = _banded(fbs, ctx, dl, dr, p, torch.from_numpy(c0).cuda(), torch.from_numpy(k0).cuda(), 0.5)
        torch.cuda.synchronize()
        fbs.fbs_sync(ctx.ctx)
    bad_learned = float(((learned - plain).abs() > 1.0).float().mean().item())
    bad_coarse = float(((coarse - plain).abs() > 1.0).float().mean().item())
    print(f"seed {seed}: threshold {thr} fallback {100 * fallback:.2f}% work {work:.3f}  extra bad px: "
          f"learned {100 * bad_learned:.3f}%  coarse {100 * bad_coarse:.3f}%")
    assert bad_learned <= 0.005
    assert work <= 0.5
    assert bad_learned < bad_coarse


def test_trained_network_beats_the_feature_point_proposal(fbs):
    """Against the paper's own future-work proposal (reliable feature points
    suggest their neighbours' range; fbs_band_feature_points, margin 0.2), at a
    similar fallback share (network threshold 0.9), the network's band leaves
    fewer extra bad pixels."""
    from synth import make_pair
    p = make_pair(WORKLOAD, 13)
    H, W, D = p.H, p.W, p.D
    with fbs.Context(0) as ctx:
        fbs.fbs_band_net_load(ctx.ctx, fbs.default_band_net_path())
        dl = torch.from_numpy(p.left).cuda()
        dr = torch.from_numpy(p.right).cuda()
        _, plain = ctx.compute_disparity(dl, dr, D, p.radius, p.sigma_s, p.sigma_r)
        c = torch.empty((H, W), device="cuda")
        k = torch.empty((H, W), device="cuda")
        fbs.fbs_band_net_forward(ctx.ctx, dl, dr, H, W, 3, D, None, c, k)
        learned = _banded(fbs, ctx, dl, dr, p, c, k, 0.9)
        fb_learned = float((k < 0.9).float().mean().item())
        fbs.fbs_band_feature_points(ctx.ctx, dl, dr, H, W, 3, D, 0.2, c, k)
        fpts = _banded(fbs, ctx, dl, dr, p, c, k, 0.5)
        fb_fp = float((k < 0.5).float().mean().item())
        torch.cuda.synchronize()
        fbs.fbs_sync(ctx.ctx)
    bad_l = float(((learned - plain).abs() > 1.0).float().mean().item())
    bad_f = float(((fpts - plain).abs() > 1.0).float().mean().item())
    print(f"learned (0.9): fallback {100 * fb_learned:.2f}% extra bad {100 * bad_l:.3f}%; "
          f"feature points (0.2): fallback {100 * fb_fp:.2f}% extra bad {100 * bad_f:.3f}%")
    assert abs(fb_learned - fb_fp) < 0.05
    assert bad_l < bad_f
