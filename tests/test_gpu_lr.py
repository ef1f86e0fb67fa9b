"""Both views and the left-right consistency check (Eq. (9)) against the oracle.

Each map follows the plain parity rules (tests/_compare.py).  The LRC decision
is an integer function of the two integer maps, so it is compared exactly
wherever neither of the winners it reads -- the left winner at (u, v) and the
right winner at (u - d, v) -- is a near tie of the oracle's aggregated costs.
"""

import numpy as np
import pytest

from tests._compare import agg_tolerance, check_disparities, near_tie_mask

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


def _run_lr(fbs, ctx, L, R, D, r, ss, sr, tau, lrc):
    H, W = L.shape[:2]
    C = L.shape[2] if L.ndim == 3 else 1
    out = [torch.empty((H, W), dtype=torch.int32, device="cuda"), torch.empty((H, W), device="cuda"),
           torch.empty((H, W), dtype=torch.int32, device="cuda"), torch.empty((H, W), device="cuda")]
    fbs.fbs_compute_disparity_lr(ctx.ctx, _dev(L), _dev(R), H, W, C, D, r, ss, sr, tau, out[0], out[1], out[2],
                                 out[3], lrc)
    torch.cuda.synchronize()
    fbs.fbs_sync(ctx.ctx)
    return [o.cpu().numpy() for o in out]


def _pair(seed, H, W, C, shift):
    rng = np.random.default_rng(seed)
    L = rng.integers(0, 256, size=(H, W, C)).astype(np.uint8)
    R = np.roll(L, -shift, axis=1)
    R = np.clip(R.astype(np.int16) + rng.integers(-5, 6, size=R.shape), 0, 255).astype(np.uint8)
    return L, R


@pytest.mark.parametrize("H,W,C,D,r,mode", [(17, 45, 3, 20, 3, 0), (24, 70, 1, 33, 4, 0), (9, 130, 3, 64, 2, 0),
                                            (13, 37, 3, 12, 2, 1), (5, 7, 3, 9, 1, 0)])
def test_both_views_and_lrc_match_the_oracle(fbs, oracle_mod, H, W, C, D, r, mode):
    L, R = _pair(H * W + D, H, W, C, shift=4)
    tau = 30.0
    with fbs.Context(0, cost=mode) as ctx:
        dl, sl, dr, sr_, = _run_lr(fbs, ctx, L, R, D, r, float(r), 12.0, tau, lrc=False)
        cl, csl, _, _ = _run_lr(fbs, ctx, L, R, D, r, float(r), 12.0, tau, lrc=True)
    rng_ = tau if mode == 1 else 2.0
    ref_l, ref_sl, agg_l = oracle_mod.fbs(L, R, D, r, float(r), 12.0, tau=tau, mode=mode, want_agg=True)
    ref_r, ref_sr, agg_r = oracle_mod.fbs_right(L, R, D, r, float(r), 12.0, tau=tau, mode=mode, want_agg=True)
    check_disparities(dl, sl, agg_l, ref_l, ref_sl, rng_)
    check_disparities(dr, sr_, agg_r, ref_r, ref_sr, rng_)
    # LRC: where both winners it reads are clear, the decision is the oracle's
    margin = 4.0 * agg_tolerance(rng_)
    tie_l = near_tie_mask(agg_l, margin)
    tie_r = near_tie_mask(agg_r, margin)
    ok_ref = oracle_mod.lrc(ref_l, ref_r)
    u = np.arange(W)[None, :].repeat(H, 0)
    ur = u - ref_l
    tie_at_match = np.zeros_like(tie_l)
    inside = ur >= 0
    tie_at_match[inside] = tie_r[np.nonzero(inside)[0], ur[inside]]
    clear = ~tie_l & ~tie_at_match
    ok_gpu = cl != -1
    assert np.array_equal(ok_gpu[clear], ok_ref[clear] == 1)
    # accepted pixels keep their disparities, rejected ones are -1 in both outputs
    assert np.array_equal(cl[ok_gpu], dl[ok_gpu]) and np.array_equal(csl[ok_gpu], sl[ok_gpu])
    assert np.all(csl[~ok_gpu] == -1.0)


def test_left_map_equals_the_single_view_entry_point(fbs):
    L, R = _pair(3, 40, 120, 3, shift=7)
    with fbs.Context(0) as ctx:
        dl, sl, _, _ = _run_lr(fbs, ctx, L, R, 32, 5, 5.0, 12.0, 0.0, lrc=False)
        di, ds = ctx.compute_disparity(_dev(L), _dev(R), 32, 5, 5.0, 12.0)
        torch.cuda.synchronize()
    assert np.array_equal(dl, di.cpu().numpy())
    assert np.array_equal(sl.view(np.uint32), ds.cpu().numpy().view(np.uint32))


def test_lrc_on_a_shifted_texture(fbs):
    """A noise-free shift by d0: the interior is confirmed and the strip with
    no match is rejected."""
    from synth import shifted_texture_pair
    H, W, D, d0, r = 32, 96, 24, 9, 3
    L, R = shifted_texture_pair(H, W, 3, d0, seed=8)
    with fbs.Context(0) as ctx:
        cl, _, dr, _ = _run_lr(fbs, ctx, L, R, D, r, 3.0, 12.0, 0.0, lrc=True)
    assert np.all(cl[r + 1:-r - 1, d0 + r + 1:-r - 1] == d0)
    assert np.all(dr[r + 1:-r - 1, r + 1:W - d0 - r - 1] == d0)
    strip = cl[:, :d0]
    assert np.mean(strip == -1) > 0.5


def test_full_size_bench_workload_row_band(fbs, oracle_mod):
    from synth import make_pair
    p = make_pair("rgb640x480_d64_r7", 0)
    with fbs.Context(0) as ctx:
        dl, sl, dr, sr_ = _run_lr(fbs, ctx, p.left, p.right, p.D, p.radius, p.sigma_s, p.sigma_r, p.tau, lrc=False)
    y0, y1 = 300, 303
    ri, rs, ragg = oracle_mod.fbs_right(p.left, p.right, p.D, p.radius, p.sigma_s, p.sigma_r, rows=(y0, y1),
                                        want_agg=True)
    check_disparities(dr[y0:y1], sr_[y0:y1], ragg, ri, rs, 2.0)


U16 = {"bf16": 2.0 ** -9, "f16": 2.0 ** -11}


@pytest.mark.parametrize("prec", ["bf16", "f16"])
@pytest.mark.parametrize("H,W,C,D,r,mode", [(17, 45, 3, 20, 3, 0), (24, 70, 1, 33, 4, 0), (13, 37, 3, 12, 2, 1)])
def test_tensor_core_both_views_match_the_oracle(fbs, oracle_mod, prec, H, W, C, D, r, mode):
    """16-bit operands: both integer maps agree with the FP64 oracle except at
    near ties of the rounding bound 3uR + 1e-5 (u the 16-bit unit roundoff,
    R the cost range), every winner is within that margin of the oracle's
    best, and the LRC decision agrees wherever both winners it reads are clear."""
    L, R = _pair(H * W + D + 7, H, W, C, shift=4)
    tau = 30.0
    p = fbs.FBS_PREC_BF16 if prec == "bf16" else fbs.FBS_PREC_F16
    with fbs.Context(0, cost=mode, prec=p) as ctx:
        dl, sl, dr, sr_ = _run_lr(fbs, ctx, L, R, D, r, float(r), 12.0, tau, lrc=False)
        cl, _, _, _ = _run_lr(fbs, ctx, L, R, D, r, float(r), 12.0, tau, lrc=True)
    rng_ = tau if mode == 1 else 2.0
    tol = 3 * U16[prec] * rng_ + 1e-5
    ref_l, _, agg_l = oracle_mod.fbs(L, R, D, r, float(r), 12.0, tau=tau, mode=mode, want_agg=True)
    ref_r, _, agg_r = oracle_mod.fbs_right(L, R, D, r, float(r), 12.0, tau=tau, mode=mode, want_agg=True)
    for di, ref, agg in ((dl, ref_l, agg_l), (dr, ref_r, agg_r)):
        ties = near_tie_mask(agg, 2 * tol)
        assert np.all((di == ref) | ties)
        chosen = np.take_along_axis(agg, di[..., None].astype(np.int64), -1)[..., 0]
        assert np.all(chosen - agg.min(-1) <= 2 * tol + 1e-12)
    clear = ~near_tie_mask(agg_l, 2 * tol)
    u = np.arange(W)[None, :].repeat(H, 0)
    ur = u - ref_l
    inside = ur >= 0
    tie_r = near_tie_mask(agg_r, 2 * tol)
    tie_at = np.zeros_like(clear)
    tie_at[inside] = tie_r[np.nonzero(inside)[0], ur[inside]]
    clear &= ~tie_at
    ok_ref = oracle_mod.lrc(ref_l, ref_r) == 1
    assert np.array_equal((cl != -1)[clear], ok_ref[clear])


def test_tensor_core_views_equal_the_single_view_path(fbs):
    """The left map is fbs_compute_disparity's; the right map is the single-view
    path on the mirrored, swapped pair, mirrored back -- both bit for bit."""
    L, R = _pair(5, 40, 120, 3, shift=7)
    with fbs.Context(0, prec=fbs.FBS_PREC_BF16) as ctx:
        dl, sl, dr, sr_ = _run_lr(fbs, ctx, L, R, 32, 5, 5.0, 12.0, 0.0, lrc=False)
        di, ds = ctx.compute_disparity(_dev(L), _dev(R), 32, 5, 5.0, 12.0)
        mi, ms = ctx.compute_disparity(_dev(R[:, ::-1]), _dev(L[:, ::-1]), 32, 5, 5.0, 12.0)
        torch.cuda.synchronize()
    assert np.array_equal(dl, di.cpu().numpy())
    assert np.array_equal(sl.view(np.uint32), ds.cpu().numpy().view(np.uint32))
    assert np.array_equal(dr, mi.cpu().numpy()[:, ::-1])
    assert np.array_equal(sr_.view(np.uint32), ms.cpu().numpy()[:, ::-1].view(np.uint32))

