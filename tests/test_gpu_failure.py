"""Failure detection without a device fault: a bounded wait that runs out, an
injected launch failure and a corrupt autotune cache, each reported through
the C ABI, with the context usable afterwards."""

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


def _pair(seed=1, H=96, W=160):
    rng = np.random.default_rng(seed)
    L = rng.integers(0, 256, size=(H, W, 3)).astype(np.uint8)
    R = np.roll(L, -6, axis=1)
    return torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()


def _run(fbs, ctx, dl, dr):
    di, ds = ctx.compute_disparity(dl, dr, 64, 7, 7.0, 12.0)
    torch.cuda.synchronize()
    return di, ds


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_wait_limit_runs_out_and_the_context_recovers(fbs, prec):
    """A limit of about 100 ns is shorter than any pipeline hand-off of the
    tensor-core aggregation, so its waits run out: the kernel stops, drains
    what it issued and frees its tensor memory, and fbs_sync reports
    FBS_ERR_TIMEOUT.  With the default limit restored the same context gives
    the results of a fresh one."""
    p = fbs.FBS_PREC_BF16 if prec == "bf16" else fbs.FBS_PREC_F16
    dl, dr = _pair()
    with fbs.Context(0, prec=p) as ref:
        di0, ds0 = _run(fbs, ref, dl, dr)
        fbs.fbs_sync(ref.ctx)
    with fbs.Context(0, prec=p) as ctx:
        fbs.fbs_set_wait_limit(ctx.ctx, 1e-7)
        _run(fbs, ctx, dl, dr)
        with pytest.raises(fbs.FBSError) as ei:
            fbs.fbs_sync(ctx.ctx)
        assert ei.value.status == fbs.FBS_ERR_TIMEOUT
        assert "bounded wait" in fbs.fbs_last_error(ctx.ctx)
        fbs.fbs_set_wait_limit(ctx.ctx, 0.0)
        di, ds = _run(fbs, ctx, dl, dr)
        fbs.fbs_sync(ctx.ctx)
        assert torch.equal(di, di0) and torch.equal(ds, ds0)
        with pytest.raises(fbs.FBSError):
            fbs.fbs_set_wait_limit(ctx.ctx, -1.0)


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_injected_launch_failure_is_reported_and_clears(fbs, prec):
    """An injected launch error surfaces as FBS_ERR_CUDA (an allocation error
    as FBS_ERR_OOM) with the error's text, launches nothing, and the next step
    runs normally."""
    p = fbs.FBS_PREC_F32 if prec == "f32" else fbs.FBS_PREC_BF16
    dl, dr = _pair(2)
    with fbs.Context(0, prec=p) as ctx:
        di0, ds0 = _run(fbs, ctx, dl, dr)
        fbs.fbs_sync(ctx.ctx)
        for err, status in ((700, fbs.FBS_ERR_CUDA), (2, fbs.FBS_ERR_OOM)):   # illegal address, memory allocation
            fbs.fbs_debug_fail_launches(ctx.ctx, err, 1)
            fbs.fbs_profile(ctx.ctx, 1)
            with pytest.raises(fbs.FBSError) as ei:
                _run(fbs, ctx, dl, dr)
            assert ei.value.status == status
            assert "injected" in fbs.fbs_last_error(ctx.ctx)
            launched = sum(fbs.fbs_profile_read(ctx.ctx, k)[1] for k in range(fbs.FBS_KERNEL_KINDS))
            fbs.fbs_profile(ctx.ctx, 0)
            assert launched == 0
            di, ds = _run(fbs, ctx, dl, dr)
            fbs.fbs_sync(ctx.ctx)
            assert torch.equal(di, di0) and torch.equal(ds, ds0)
        with pytest.raises(fbs.FBSError):
            fbs.fbs_debug_fail_launches(ctx.ctx, 0, 1)


def test_corrupt_autotune_cache_is_ignored(fbs, tmp_path):
    """Garbage, out-of-range plans and truncated lines in the autotune cache
    file are skipped: the batch still runs (autotuned afresh), gives the
    per-pair results, and a valid entry is appended."""
    from synth import random_batch_specs
    path = tmp_path / "tune.txt"
    path.write_bytes(b"\x00\xff garbage line\nt64x2 99\nf1 -3\nnot_a_number x\nt12")
    specs = random_batch_specs(11, n=3, wrange=(64, 128), hrange=(48, 96), dchoices=(16, 32), rchoices=(2, 4))
    pairs, ref = [], []
    with fbs.Context(0, prec=fbs.FBS_PREC_BF16, autotune_cache_path=str(path)) as ctx:
        for sp in specs:
            rng = np.random.default_rng(sp["seed"])
            L = rng.integers(0, 256, size=(sp["H"], sp["W"], 3)).astype(np.uint8)
            R = np.roll(L, -3, axis=1)
            dl, dr = torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()
            q = dict(left=dl, right=dr, H=sp["H"], W=sp["W"], C=3, D=sp["D"], radius=sp["radius"],
                     sigma_s=sp["sigma_s"], sigma_r=12.0, tau=30.0,
                     disp_int=torch.empty((sp["H"], sp["W"]), dtype=torch.int32, device="cuda"),
                     disp_subpix=torch.empty((sp["H"], sp["W"]), dtype=torch.float32, device="cuda"))
            pairs.append(q)
            di, ds = ctx.compute_disparity(dl, dr, sp["D"], sp["radius"], sp["sigma_s"], 12.0, 30.0)
            ref.append((di, ds))
        assert fbs.fbs_batch_plan(ctx.ctx, pairs) == -1
        fbs.fbs_compute_disparity_batched(ctx.ctx, pairs, torch.cuda.current_stream())
        torch.cuda.synchronize()
        fbs.fbs_sync(ctx.ctx)
        plan = fbs.fbs_batch_plan(ctx.ctx, pairs)
        assert plan >= 0
        for q, (di, ds) in zip(pairs, ref):
            assert torch.equal(q["disp_int"], di) and torch.equal(q["disp_subpix"], ds)
    last = path.read_bytes().splitlines()[-1].split()
    assert len(last) == 2 and int(last[1]) == plan
