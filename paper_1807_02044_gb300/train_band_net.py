"""Train the band-proposal network of the learned band form on the GPU.

Training pairs are seeded synthetic stereo pairs of the 1920x1080 RGB,
D = 256, radius 9 workload: ``--scenes`` scenes rendered by ``synth`` (in a
spawned process pool, while the GPU trains), each cut into random crops of
``--crop`` pixels; a crop of both views at the same rows and columns is itself
a stereo pair of the scene, so ``--pairs`` crops give that many distinct
pairs.  Each pair is labelled by the plain full-range path (FP32) and used for
one training step (forward, loss, backward, Adam) -- all in libfbs's own
kernels.  The step size follows a cosine schedule from ``--lr`` to lr/20.

Held-out scenes (other seeds) measure, at full size, what the trained network
gives the band path: the extra bad-pixel rate (> 1 px) against the plain
path, the fraction of pixels falling back to the full range, and the
fraction of the full-range aggregation work that remains.

    python -m paper_1807_02044_gb300.train_band_net --out band_net.bin
"""

from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import math
import multiprocessing as mp
import os
import sys
import time
import types

import numpy as np

WORKLOAD = "rgb1920x1080_d256_r9"
HALF_BAND = 8
THRESHOLDS = (0.5, 0.8, 0.9, 0.95, 0.98, 0.985, 0.99, 0.9925, 0.995, 0.9975)
TARGET_EXTRA_BAD_PCT = 0.47     # chosen threshold: mean extra bad pixels below this on the held-out scenes


def _render(seed):
    from synth import make_pair
    p = make_pair(WORKLOAD, seed)
    return seed, p.left, p.right, p.gt, p.occ


def band_metrics(fbs, ctx, dl, dr, p, thresholds=THRESHOLDS, half_band=HALF_BAND, gt=None, occ=None):
    """Plain vs learned band path on one full pair (device images dl, dr), for
    each confidence threshold: extra bad pixels (> 1 px against the plain
    path), pixels falling back to the full range, and the remaining fraction
    of the full-range aggregation work; with the scene's ground truth also the
    bad-pixel rates (> 1 px against it, unoccluded pixels) of both paths."""
    import torch
    H, W, D = p.H, p.W, p.D
    st = torch.cuda.current_stream(dl.device)   # every call below on this one stream
    di, ds = ctx.compute_disparity(dl, dr, D, p.radius, p.sigma_s, p.sigma_r, stream=st)
    centre = torch.empty((H, W), device=dl.device)
    conf = torch.empty((H, W), device=dl.device)
    fbs.fbs_band_net_forward(ctx.ctx, dl, dr, H, W, 3, D, None, centre, conf, st)
    bi = torch.empty((H, W), dtype=torch.int32, device=dl.device)
    bs = torch.empty((H, W), device=dl.device)
    lo = torch.empty((H, W), dtype=torch.int32, device=dl.device)
    hi = torch.empty((H, W), dtype=torch.int32, device=dl.device)
    out = []
    bad_gt = None
    if gt is not None:
        gtd = torch.from_numpy(gt).to(dl.device)
        vis = torch.from_numpy(~occ).to(dl.device)
        bad_gt = lambda d: 100.0 * (((d - gtd).abs() > 1.0) & vis).double().sum().item() / vis.sum().item()
    for th in thresholds:
        fbs.fbs_compute_disparity_banded(ctx.ctx, dict(left=dl, right=dr, H=H, W=W, C=3, D=D, radius=p.radius,
                                                       sigma_s=p.sigma_s, sigma_r=p.sigma_r, disp_int=bi,
                                                       disp_subpix=bs), centre, conf, half_band, th, st)
        fbs.fbs_band_limits(ctx.ctx, centre, conf, H * W, D, half_band, th, lo, hi, st)
        torch.cuda.synchronize()
        fbs.fbs_sync(ctx.ctx)
        out.append(dict(threshold=th, extra_bad_pct=100.0 * ((bs - ds).abs() > 1.0).float().mean().item(),
                        fallback_pct=100.0 * (conf < th).float().mean().item(),
                        work_fraction=((hi - lo + 1).double().sum() / (H * W * D)).item()))
        if bad_gt is not None:
            out[-1].update(bad_vs_gt_pct=bad_gt(bs), plain_bad_vs_gt_pct=bad_gt(ds))
    return out


def choose_threshold(sweep, target=TARGET_EXTRA_BAD_PCT):
    """The smallest threshold whose mean extra bad-pixel rate (against the
    plain path) is at most `target` percent on the held-out scenes."""
    ok = [r for r in sweep if r["extra_bad_pct"] <= target]
    return ok[0]["threshold"] if ok else sweep[-1]["threshold"]


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--out", required=True, help="weights file to write")
    ap.add_argument("--summary", default=None, help="JSON file for the training record")
    ap.add_argument("--pairs", type=int, default=10000)
    ap.add_argument("--scenes", type=int, default=400)
    ap.add_argument("--crop", default="1280x640", help="crop W x H of each training pair")
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0, help="network initialisation and crop positions")
    ap.add_argument("--scene-seed0", type=int, default=100000, help="first scene seed of the training set")
    ap.add_argument("--val-scenes", type=int, default=6)
    ap.add_argument("--workers", type=int, default=0)
    args = ap.parse_args(argv)

    cw, ch = (int(v) for v in args.crop.lower().split("x"))
    workers = args.workers or max(1, (os.cpu_count() or 2) - 1)
    per_scene = math.ceil(args.pairs / args.scenes)
    train_seeds = list(range(args.scene_seed0, args.scene_seed0 + args.scenes))
    val_seeds = list(range(args.scene_seed0 - args.val_scenes, args.scene_seed0))

    # the pool is spawned before the first GPU call
    pool = cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
    import torch

    import paper_1807_02044_gb300 as fbs
    from synth import WORKLOADS
    spec = WORKLOADS[WORKLOAD]
    D, radius, ss, sr = spec["D"], spec["radius"], spec["sigma_s"], spec["sigma_r"]
    rng = np.random.default_rng(args.seed)
    st = torch.cuda.current_stream()   # crops, labels and training steps are ordered on this stream
    log = []
    t0 = time.time()
    with fbs.Context(0) as ctx:
        fbs.fbs_band_net_init(ctx.ctx, args.seed)
        torch.cuda.synchronize()
        step = 0
        for seed, L, R, _, _ in pool.map(_render, train_seeds):
            dl = torch.from_numpy(L).cuda()
            dr = torch.from_numpy(R).cuda()
            H, W = L.shape[:2]
            for _ in range(per_scene):
                if step >= args.pairs:
                    break
                y0 = int(rng.integers(0, H - ch + 1))
                x0 = int(rng.integers(0, W - cw + 1))
                cl = dl[y0:y0 + ch, x0:x0 + cw].contiguous()
                cr = dr[y0:y0 + ch, x0:x0 + cw].contiguous()
                li, ls = ctx.compute_disparity(cl, cr, D, radius, ss, sr, stream=st)
                lr = args.lr * (0.05 + 0.95 * 0.5 * (1.0 + math.cos(math.pi * step / args.pairs)))
                want = step % 100 == 0 or step == args.pairs - 1
                loss = np.zeros(1, np.float32) if want else None
                fbs.fbs_band_net_train_step(ctx.ctx, cl, cr, ch, cw, 3, D, li, ls, HALF_BAND, lr, loss, None, st)
                if want:
                    log.append(dict(step=step, scene=seed, loss=float(loss[0]), lr=lr,
                                    seconds=round(time.time() - t0, 1)))
                    print(json.dumps(log[-1]), flush=True)
                step += 1
            if step >= args.pairs:
                break
        fbs.fbs_band_net_save(ctx.ctx, args.out)
        train_s = time.time() - t0
        val = []
        for seed, L, R, gt, occ in pool.map(_render, val_seeds):
            dl = torch.from_numpy(L).cuda()
            dr = torch.from_numpy(R).cuda()
            q = types.SimpleNamespace(H=L.shape[0], W=L.shape[1], D=D, radius=radius, sigma_s=ss, sigma_r=sr)
            m = band_metrics(fbs, ctx, dl, dr, q, gt=gt.astype(np.float32), occ=occ)
            val.append(dict(scene=seed, thresholds=m))
            print(json.dumps(val[-1]), flush=True)
    pool.shutdown()
    # the smallest threshold whose mean extra bad-pixel rate stays under the target
    sweep = []
    for i, th in enumerate(THRESHOLDS):
        rows = [v["thresholds"][i] for v in val]
        sweep.append(dict(threshold=th, **{k: float(np.mean([r[k] for r in rows]))
                                           for k in ("extra_bad_pct", "fallback_pct", "work_fraction",
                                                     "bad_vs_gt_pct", "plain_bad_vs_gt_pct")}))
    chosen = choose_threshold(sweep)
    summary = dict(workload=WORKLOAD, pairs=step, scenes=len(train_seeds), crop=[cw, ch], half_band=HALF_BAND,
                   threshold=chosen, target_extra_bad_pct=TARGET_EXTRA_BAD_PCT, lr=args.lr, seed=args.seed,
                   scene_seeds=[train_seeds[0], train_seeds[-1]], val_seeds=val_seeds,
                   train_seconds=round(train_s, 1), validation_mean=sweep, validation=val, loss_log=log,
                   command="python -m paper_1807_02044_gb300.train_band_net " + " ".join(sys.argv[1:]))
    if args.summary:
        with open(args.summary, "w") as f:
            json.dump(summary, f, indent=1)
    return summary


if __name__ == "__main__":
    main()
