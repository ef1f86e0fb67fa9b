"""fbs_compute_disparity_noalloc against fbs_compute_disparity, through the C ABI.

The no-allocation entry point serves callers that cannot call cudaMalloc
while they run (a plugin whose host application owns all device memory, a
real-time loop with a memory budget fixed at start-up).  It keeps the cost
volume in the library's fixed static scratch instead of the context's
scratch, so its results must match the allocating entry point's.  This file
is named to be collected last, so a failure here does not hide the other
tests in a run that stops at the first failure.
"""

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


def _pair(H, W, C, D, seed):
    rng = np.random.default_rng(seed)
    L = rng.integers(0, 256, size=(H, W, C)).astype(np.uint8)
    R = np.roll(L, -min(D // 2, W - 1), axis=1)
    return torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()


def _run_both(fbs, ctx, L, R, H, W, C, D, r, tau, stream):
    di_ref = torch.empty((H, W), dtype=torch.int32, device="cuda")
    ds_ref = torch.empty((H, W), dtype=torch.float32, device="cuda")
    fbs.fbs_compute_disparity(ctx.ctx, L, R, H, W, C, D, r, float(r), 12.0, tau, di_ref, ds_ref, stream)
    di = torch.full((H, W), -1, dtype=torch.int32, device="cuda")
    ds = torch.full((H, W), -1.0, dtype=torch.float32, device="cuda")
    fbs.fbs_compute_disparity_noalloc(ctx.ctx, L, R, H, W, C, D, r, float(r), 12.0, tau, di, ds, stream)
    torch.cuda.synchronize()
    return di_ref, ds_ref, di, ds


@pytest.mark.parametrize("cost,tau", [("NCC", 0.0), ("TAD", 40.0)])
def test_noalloc_matches_allocating_entry_point_on_consecutive_calls(fbs, cost, tau):
    """Both entry points run the same kernels on the same inputs, so integer
    and subpixel maps are identical bit for bit, for NCC and TAD costs."""
    ctx = fbs.Context(0, cost=getattr(fbs, "FBS_COST_" + cost))
    try:
        stream = torch.cuda.current_stream()
        # calls in a row, each smaller than the one before, so stale contents
        # of the shared scratch would show up if they were read; the first
        # nearly fills it (D=104 is the largest that fits at 320x240)
        for (H, W, C, D, r), seed in [((240, 320, 3, 104, 5), 4), ((120, 160, 1, 16, 4), 1),
                                      ((61, 97, 3, 20, 3), 2)]:
            L, R = _pair(H, W, C, D, seed)
            di_ref, ds_ref, di, ds = _run_both(fbs, ctx, L, R, H, W, C, D, r, tau, stream)
            assert torch.equal(di, di_ref)
            assert torch.equal(ds, ds_ref)
    finally:
        ctx.close()


def test_noalloc_counts_and_times_its_kernels(fbs):
    """The kernels count under FBS_KERNEL_COST (statistics pre-pass and cost
    kernel) and FBS_KERNEL_AGG_F32 and are timed when profiling is on."""
    H, W, C, D, r = 96, 128, 3, 24, 3
    ctx = fbs.Context(0)
    try:
        L, R = _pair(H, W, C, D, 5)
        di = torch.empty((H, W), dtype=torch.int32, device="cuda")
        fbs.fbs_compute_disparity_noalloc(ctx.ctx, L, R, H, W, C, D, r, 3.0, 12.0, 0.0, di, None, None)
        fbs.fbs_sync(ctx.ctx)
        fbs.fbs_profile(ctx.ctx, 1)
        for _ in range(2):
            fbs.fbs_compute_disparity_noalloc(ctx.ctx, L, R, H, W, C, D, r, 3.0, 12.0, 0.0, di, None, None)
        fbs.fbs_sync(ctx.ctx)
        ms_c, n_c = fbs.fbs_profile_read(ctx.ctx, fbs.FBS_KERNEL_COST)
        ms_a, n_a = fbs.fbs_profile_read(ctx.ctx, fbs.FBS_KERNEL_AGG_F32)
        fbs.fbs_profile(ctx.ctx, 0)
        assert (n_c, n_a) == (4, 2)
        assert ms_c > 0 and ms_a > 0
    finally:
        ctx.close()


def test_noalloc_reports_launch_failures_like_the_allocating_path(fbs):
    """An injected launch failure returns FBS_ERR_CUDA, an injected
    out-of-memory error FBS_ERR_OOM, and neither launches anything."""
    H, W, C, D = 32, 48, 3, 8
    ctx = fbs.Context(0)
    try:
        L, R = _pair(H, W, C, D, 6)
        di = torch.empty((H, W), dtype=torch.int32, device="cuda")
        fbs.fbs_profile(ctx.ctx, 1)
        for err, status in [(700, fbs.FBS_ERR_CUDA), (2, fbs.FBS_ERR_OOM)]:
            fbs.fbs_debug_fail_launches(ctx.ctx, err, 1)
            with pytest.raises(fbs.FBSError) as ei:
                fbs.fbs_compute_disparity_noalloc(ctx.ctx, L, R, H, W, C, D, 2, 2.0, 12.0, 0.0, di, None, None)
            assert ei.value.status == status
        counts = [fbs.fbs_profile_read(ctx.ctx, k)[1] for k in range(fbs.FBS_KERNEL_KINDS)]
        assert counts == [0] * fbs.FBS_KERNEL_KINDS
        # the context works again once the injected failures are used up
        fbs.fbs_compute_disparity_noalloc(ctx.ctx, L, R, H, W, C, D, 2, 2.0, 12.0, 0.0, di, None, None)
        fbs.fbs_sync(ctx.ctx)
        fbs.fbs_profile(ctx.ctx, 0)
    finally:
        ctx.close()


def test_noalloc_rejects_sizes_beyond_its_static_scratch(fbs):
    """Requests one disparity beyond the limit fail before any launch; the
    images and outputs are full size, so a launch could not go out of bounds
    even if one happened."""
    ctx = fbs.Context(0)
    try:
        fbs.fbs_profile(ctx.ctx, 1)
        for H, W, C, D in [(480, 640, 3, 24), (240, 320, 1, 105), (480, 640, 3, 64)]:
            assert H * W * (4 * ((D + 3) // 4 * 4) + 20) > fbs.FBS_NOALLOC_MAX_COST_BYTES
            L, R = _pair(H, W, C, D, 3)
            out = torch.empty((H, W), dtype=torch.int32, device="cuda")
            with pytest.raises(fbs.FBSError) as ei:
                fbs.fbs_compute_disparity_noalloc(ctx.ctx, L, R, H, W, C, D, 7, 7.0, 12.0, 0.0, out, None, None)
            assert ei.value.status == fbs.FBS_ERR_INVALID_ARG
            assert "exceeds the static scratch" in str(ei.value)
        fbs.fbs_sync(ctx.ctx)
        counts = [fbs.fbs_profile_read(ctx.ctx, k)[1] for k in range(fbs.FBS_KERNEL_KINDS)]
        assert counts == [0] * fbs.FBS_KERNEL_KINDS
        fbs.fbs_profile(ctx.ctx, 0)
    finally:
        ctx.close()
