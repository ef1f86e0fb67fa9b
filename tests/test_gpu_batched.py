"""Batched form through the C ABI: uneven pairs in one CUDA graph must
reproduce fbs_compute_disparity bit for bit in the context's precision (FP32:
one persistent launch per stage, same tile code, same data, same order;
BF16 / FP16: the single-pair tensor-core launches spread over concurrent graph
branches, or the cost builds and one persistent tensor-core launch over the
tiles of every pair), under every plan, and the autotuner's choice must
persist."""

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fbs():
    from paper_1807_02044_gb300 import build as b
    b.build()
    import paper_1807_02044_gb300 as m
    return m


def _batch(seed, n=9):
    rng = np.random.default_rng(seed)
    pairs = []
    for i in range(n):
        H, W = int(rng.integers(20, 90)), int(rng.integers(33, 160))
        C = int(rng.choice([1, 3]))
        D = int(rng.choice([8, 16, 21, 32, 40, 70]))
        r = int(rng.choice([0, 1, 2, 4, 7]))
        L = rng.integers(0, 256, size=(H, W, C)).astype(np.uint8)
        R = np.roll(L, -int(rng.integers(0, 6)), axis=1)
        pairs.append(dict(left=torch.from_numpy(L).cuda(), right=torch.from_numpy(R).cuda(), H=H, W=W, C=C, D=D,
                          radius=r, sigma_s=float(max(r, 1)), sigma_r=12.0, tau=20.0,
                          disp_int=torch.empty((H, W), dtype=torch.int32, device="cuda"),
                          disp_subpix=torch.empty((H, W), dtype=torch.float32, device="cuda")))
    return pairs


@pytest.mark.parametrize("mode", [0, 1])
def test_batched_equals_per_pair_bit_for_bit(fbs, mode):
    pairs = _batch(3 + mode)
    with fbs.Context(0, cost=mode) as ctx:
        ref = []
        for q in pairs:
            di, ds = ctx.compute_disparity(q["left"], q["right"], q["D"], q["radius"], q["sigma_s"], q["sigma_r"],
                                           q["tau"])
            ref.append((di, ds))
        torch.cuda.synchronize()
        fbs.fbs_compute_disparity_batched(ctx.ctx, pairs, torch.cuda.current_stream())
        torch.cuda.synchronize()
        fbs.fbs_sync(ctx.ctx)
        for q, (di, ds) in zip(pairs, ref):
            assert torch.equal(q["disp_int"], di)
            assert torch.equal(q["disp_subpix"], ds)
        plan = fbs.fbs_batch_plan(ctx.ctx, pairs)
        assert 0 <= plan < 7
        # replay with fresh output buffers and new images of the same shapes
        pairs2 = _batch(3 + mode)
        for q in pairs2:
            q["left"] = torch.flip(q["left"], dims=[0]).contiguous()
        fbs.fbs_compute_disparity_batched(ctx.ctx, pairs2, torch.cuda.current_stream())
        for q in pairs2:
            di, ds = ctx.compute_disparity(q["left"], q["right"], q["D"], q["radius"], q["sigma_s"], q["sigma_r"],
                                           q["tau"])
            torch.cuda.synchronize()
            assert torch.equal(q["disp_int"], di)
            assert torch.equal(q["disp_subpix"], ds)


def test_batched_matches_oracle_on_a_member(fbs, oracle_mod):
    from tests._compare import check_disparities
    pairs = _batch(11, n=4)
    with fbs.Context(0) as ctx:
        fbs.fbs_compute_disparity_batched(ctx.ctx, pairs, torch.cuda.current_stream())
        torch.cuda.synchronize()
    for q in pairs:
        L, R = q["left"].cpu().numpy(), q["right"].cpu().numpy()
        ref_di, ref_ds, ref_agg = oracle_mod.fbs(L, R, q["D"], q["radius"], q["sigma_s"], q["sigma_r"], want_agg=True)
        check_disparities(q["disp_int"].cpu().numpy(), q["disp_subpix"].cpu().numpy(), ref_agg, ref_di, ref_ds, 2.0)


def test_autotune_choice_is_stored_and_reloaded(fbs, tmp_path):
    path = str(tmp_path / "tune.txt")
    pairs = _batch(5, n=5)
    with fbs.Context(0, autotune_cache_path=path) as ctx:
        assert fbs.fbs_batch_plan(ctx.ctx, pairs) == -1
        fbs.fbs_compute_disparity_batched(ctx.ctx, pairs, torch.cuda.current_stream())
        torch.cuda.synchronize()
        plan = fbs.fbs_batch_plan(ctx.ctx, pairs)
    assert os.path.exists(path) and open(path).read().strip().endswith(str(plan))
    with fbs.Context(0, autotune_cache_path=path) as ctx2:
        assert fbs.fbs_batch_plan(ctx2.ctx, pairs) == plan


def test_batched_rejects_bad_pairs(fbs):
    pairs = _batch(7, n=3)
    pairs[1]["radius"] = 40
    with fbs.Context(0) as ctx:
        with pytest.raises(fbs.FBSError) as ei:
            fbs.fbs_compute_disparity_batched(ctx.ctx, pairs)
        assert ei.value.status == fbs.FBS_ERR_INVALID_ARG and "pair 1" in str(ei.value)
        ctx.set_options(prec=fbs.FBS_PREC_BF16)
        pairs[1]["radius"] = 2
        pairs[2]["D"] = 300   # beyond the tensor-core form's 256
        with pytest.raises(fbs.FBSError) as ei:
            fbs.fbs_compute_disparity_batched(ctx.ctx, pairs)
        assert ei.value.status == fbs.FBS_ERR_UNSUPPORTED and "pair 2" in str(ei.value)
        with pytest.raises(fbs.FBSError) as ei:
            fbs.fbs_batch_set_plan(ctx.ctx, pairs, 7)
        assert ei.value.status == fbs.FBS_ERR_INVALID_ARG


@pytest.mark.parametrize("mode", [0, 1])
def test_fp32_batch_equals_per_pair_under_every_plan(fbs, mode):
    """Persistent plans 0-3 and branched plans 4-6."""
    pairs = _batch(41 + mode, n=7)
    with fbs.Context(0, cost=mode) as ctx:
        ref = _per_pair(ctx, pairs)
        for plan in range(7):
            for q in pairs:
                q["disp_int"].fill_(-7)
                q["disp_subpix"].fill_(-7.0)
            fbs.fbs_batch_set_plan(ctx.ctx, pairs, plan)
            fbs.fbs_compute_disparity_batched(ctx.ctx, pairs, torch.cuda.current_stream())
            torch.cuda.synchronize()
            fbs.fbs_sync(ctx.ctx)
            for i, (q, (di, ds)) in enumerate(zip(pairs, ref)):
                assert torch.equal(q["disp_int"], di), (plan, i)
                assert torch.equal(q["disp_subpix"], ds), (plan, i)
        with pytest.raises(fbs.FBSError):
            fbs.fbs_batch_set_plan(ctx.ctx, pairs, 7)


def _tc_variants(pairs):
    """Radius variants of the tensor-core producers in a batch: the persistent
    plan launches one aggregation per variant (column pairs per thread
    ceil((r + 1) / 2) exact up to 8, split by the parity of r; 10 and 13
    above)."""
    def v(r):
        npt = (r + 2) // 2
        return (npt, r & 1) if npt <= 8 else (10 if npt <= 10 else 13,)
    return len({v(q["radius"]) for q in pairs})


def _per_pair(ctx, pairs):
    ref = []
    for q in pairs:
        ref.append(ctx.compute_disparity(q["left"], q["right"], q["D"], q["radius"], q["sigma_s"], q["sigma_r"],
                                         q["tau"]))
    torch.cuda.synchronize()
    return ref


@pytest.mark.parametrize("prec,mode", [("bf16", 0), ("fp16", 0), ("bf16", 1)])
def test_tensor_core_batch_equals_per_pair_under_every_plan(fbs, prec, mode):
    p = fbs.FBS_PREC_BF16 if prec == "bf16" else fbs.FBS_PREC_F16
    pairs = _batch(21 + mode, n=11)
    pairs[0]["D"], pairs[0]["radius"] = 256, 9    # the largest disparity range, more than one TMEM block
    with fbs.Context(0, cost=mode, prec=p) as ctx:
        ref = _per_pair(ctx, pairs)
        for plan in range(7):
            for q in pairs:
                q["disp_int"].fill_(-7)
                q["disp_subpix"].fill_(-7.0)
            fbs.fbs_batch_set_plan(ctx.ctx, pairs, plan)
            assert fbs.fbs_batch_plan(ctx.ctx, pairs) == plan
            fbs.fbs_compute_disparity_batched(ctx.ctx, pairs, torch.cuda.current_stream())
            torch.cuda.synchronize()
            fbs.fbs_sync(ctx.ctx)
            for i, (q, (di, ds)) in enumerate(zip(pairs, ref)):
                assert torch.equal(q["disp_int"], di), (plan, i)
                assert torch.equal(q["disp_subpix"], ds), (plan, i)


def test_tensor_core_batch_autotunes_and_follows_new_buffers(fbs):
    pairs = _batch(31, n=6)
    with fbs.Context(0, prec=fbs.FBS_PREC_BF16) as ctx:
        assert fbs.fbs_batch_plan(ctx.ctx, pairs) == -1
        fbs.fbs_profile(ctx.ctx, 1)
        fbs.fbs_compute_disparity_batched(ctx.ctx, pairs, torch.cuda.current_stream())
        torch.cuda.synchronize()
        plan = fbs.fbs_batch_plan(ctx.ctx, pairs)
        assert 0 <= plan < 7
        ref = _per_pair(ctx, pairs)
        for q, (di, ds) in zip(pairs, ref):
            assert torch.equal(q["disp_int"], di) and torch.equal(q["disp_subpix"], ds)
        # every kernel is counted: per pair one cost kernel, and one aggregation
        # per pair or (plan 6) one persistent aggregation per radius variant
        fbs.fbs_profile(ctx.ctx, 1)
        fbs.fbs_compute_disparity_batched(ctx.ctx, pairs, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert fbs.fbs_profile_read(ctx.ctx, fbs.FBS_KERNEL_AGG_TC)[1] == (_tc_variants(pairs) if plan == 6
                                                                           else len(pairs))
        assert fbs.fbs_profile_read(ctx.ctx, fbs.FBS_KERNEL_COST)[1] == len(pairs)
        fbs.fbs_profile(ctx.ctx, 0)
        # new output buffers and new images of the same shapes: a new graph, the same results as per-pair calls
        pairs2 = _batch(31, n=6)
        for q in pairs2:
            q["left"] = torch.flip(q["left"], dims=[1]).contiguous()
        fbs.fbs_compute_disparity_batched(ctx.ctx, pairs2, torch.cuda.current_stream())
        torch.cuda.synchronize()
        got = [(q["disp_int"].clone(), q["disp_subpix"].clone()) for q in pairs2]
        ref2 = _per_pair(ctx, pairs2)
        for (gi, gs), (di, ds) in zip(got, ref2):
            assert torch.equal(gi, di) and torch.equal(gs, ds)
        fbs.fbs_sync(ctx.ctx)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_persistent_tensor_core_plan_covers_every_radius_variant(fbs, prec):
    """Plan 6 (persistent tensor-core launches over every pair's tiles) on
    a batch whose radii reach every instantiated column-pair variant (radius
    0 .. 24, odd and even, including the two generic wide ones) and whose
    disparity ranges span one to more than one TMEM block (D up to 256, where
    the normaliser takes its own MMA): bit-identical to per-pair calls."""
    p = fbs.FBS_PREC_BF16 if prec == "bf16" else fbs.FBS_PREC_F16
    rng = np.random.default_rng(77)
    radii = list(range(0, 17)) + [17, 19, 20, 22, 24]
    Ds = [8, 16, 24, 40, 64, 100, 128, 200, 256]
    pairs = []
    for i, r in enumerate(radii):
        H, W = int(rng.integers(9, 70)), int(rng.integers(17, 120))
        C = int(rng.choice([1, 3]))
        D = Ds[i % len(Ds)]
        L = rng.integers(0, 256, size=(H, W, C)).astype(np.uint8)
        R = np.roll(L, -int(rng.integers(0, 6)), axis=1)
        pairs.append(dict(left=torch.from_numpy(L).cuda(), right=torch.from_numpy(R).cuda(), H=H, W=W, C=C, D=D,
                          radius=r, sigma_s=float(max(r, 1)), sigma_r=12.0, tau=20.0,
                          disp_int=torch.full((H, W), -7, dtype=torch.int32, device="cuda"),
                          disp_subpix=torch.full((H, W), -7.0, dtype=torch.float32, device="cuda")))
    with fbs.Context(0, prec=p) as ctx:
        ref = _per_pair(ctx, pairs)
        fbs.fbs_batch_set_plan(ctx.ctx, pairs, 6)
        fbs.fbs_profile(ctx.ctx, 1)
        for rep in range(2):   # the second call replays the same graph
            fbs.fbs_compute_disparity_batched(ctx.ctx, pairs, torch.cuda.current_stream())
            torch.cuda.synchronize()
            fbs.fbs_sync(ctx.ctx)
            for i, (q, (di, ds)) in enumerate(zip(pairs, ref)):
                assert torch.equal(q["disp_int"], di), (rep, i, q["radius"], q["D"])
                assert torch.equal(q["disp_subpix"], ds), (rep, i, q["radius"], q["D"])
        assert fbs.fbs_profile_read(ctx.ctx, fbs.FBS_KERNEL_AGG_TC)[1] == 2 * _tc_variants(pairs) == 2 * 18
        fbs.fbs_profile(ctx.ctx, 0)


def test_persistent_tensor_core_plan_member_matches_oracle(fbs, oracle_mod):
    """A BF16 member of the persistent plan against the FP64 oracle: integer
    and subpixel disparities under the 16-bit rules (aggregated-cost bound
    3 u R + 1e-5, u = 2^-9, R = 2)."""
    from tests._compare import check_disparities
    pairs = _batch(13, n=5)
    with fbs.Context(0, prec=fbs.FBS_PREC_BF16) as ctx:
        fbs.fbs_batch_set_plan(ctx.ctx, pairs, 6)
        fbs.fbs_compute_disparity_batched(ctx.ctx, pairs, torch.cuda.current_stream())
        torch.cuda.synchronize()
        fbs.fbs_sync(ctx.ctx)
    tol = 3 * 2.0 ** -9 * 2.0 + 1e-5
    for q in pairs:
        L, R = q["left"].cpu().numpy(), q["right"].cpu().numpy()
        ref_di, ref_ds, ref_agg = oracle_mod.fbs(L, R, q["D"], q["radius"], q["sigma_s"], q["sigma_r"], want_agg=True)
        check_disparities(q["disp_int"].cpu().numpy(), q["disp_subpix"].cpu().numpy(), ref_agg, ref_di, ref_ds, 2.0,
                          tol=tol)
