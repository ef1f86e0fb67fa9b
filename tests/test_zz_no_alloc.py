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

from tests._compare import SUBPIX_TOL

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


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls(fbs):
    ctx = fbs.Context(0)
    try:
        stream = torch.cuda.current_stream()
        # two calls in a row, the second smaller than the first so stale
        # contents of the shared scratch would show up if they were read
        for (H, W, C, D, r), seed in [((120, 160, 1, 16, 4), 1), ((61, 97, 3, 20, 3), 2)]:
            L, R = _pair(H, W, C, D, seed)
            di_ref = torch.empty((H, W), dtype=torch.int32, device="cuda")
            ds_ref = torch.empty((H, W), dtype=torch.float32, device="cuda")
            fbs.fbs_compute_disparity(ctx.ctx, L, R, H, W, C, D, r, float(r), 12.0, 0.0, di_ref, ds_ref, stream)
            di = torch.full((H, W), -1, dtype=torch.int32, device="cuda")
            ds = torch.full((H, W), -1.0, dtype=torch.float32, device="cuda")
            fbs.fbs_compute_disparity_noalloc(ctx.ctx, L, R, H, W, C, D, r, float(r), 12.0, 0.0, di, ds, stream)
            torch.cuda.synchronize()
            assert torch.equal(di, di_ref)
            assert float((ds - ds_ref).abs().max()) <= SUBPIX_TOL
    finally:
        ctx.close()


def test_noalloc_rejects_sizes_beyond_its_static_scratch(fbs):
    ctx = fbs.Context(0)
    try:
        H, W, D = 480, 640, 64          # 78.6 MB of cost volume > the fixed scratch
        assert H * W * D * 4 > fbs.FBS_NOALLOC_MAX_COST_BYTES
        L, R = _pair(8, 8, 3, 4, 3)
        out = torch.empty((H, W), dtype=torch.int32, device="cuda")
        with pytest.raises(fbs.FBSError) as ei:
            fbs.fbs_compute_disparity_noalloc(ctx.ctx, L, R, H, W, 3, D, 7, 7.0, 12.0, 0.0, out, None)
        assert ei.value.status == fbs.FBS_ERR_INVALID_ARG
        assert "exceeds the static scratch" in str(ei.value)
    finally:
        ctx.close()
