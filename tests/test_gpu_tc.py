"""Tensor-core (BF16 / FP16 operand) aggregation through the C ABI.

Tolerances come from the arithmetic: with unit roundoff u of the 16-bit type
(2^-9 for BF16, 2^-11 for FP16) applied to every cost and every weight, and
the normaliser summed from the same rounded weights in FP32,
    |Agg_tc - Agg| <= u max|C| + 2u max|C - Agg| / (1 - u) + FP32 terms
                   <= 3 u R + 1e-5          (R = cost range = 2 for NCC).
"""

import numpy as np
import pytest

from tests._compare import check_disparities, near_tie_mask

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = {"bf16": 2.0 ** -9, "f16": 2.0 ** -11}


@pytest.fixture(scope="module")
def fbs():
    from paper_1807_02044_gb300 import build as b
    b.build()
    import paper_1807_02044_gb300 as m
    return m


def _prec(fbs, name):
    return fbs.FBS_PREC_BF16 if name == "bf16" else fbs.FBS_PREC_F16


def _round16(a, name):
    t = torch.from_numpy(np.ascontiguousarray(a, np.float32))
    return (t.to(torch.bfloat16) if name == "bf16" else t.to(torch.float16)).to(torch.float32).numpy()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("prec", ["bf16", "f16"])
@pytest.mark.parametrize("H,W,D", [(8, 16, 16), (13, 37, 20), (24, 50, 64), (9, 40, 250), (10, 24, 256)])
def test_radius_zero_returns_the_rounded_cost_exactly(fbs, prec, H, W, D):
    """With radius 0 every pixel's only weight is 1, so the tensor-core product
    must reproduce the 16-bit cost bit for bit: this pins the operand layouts,
    the TMA box, the instruction descriptor and the accumulator read-out
    (D > 240: the two MMAs of N = 128 and N - 128 per K-step)."""
    rng = np.random.default_rng(H * W + D)
    cost = (rng.random((H, W, D)) * 2).astype(np.float32)
    G = rng.integers(0, 256, size=(H, W, 3)).astype(np.uint8)
    with fbs.Context(0, prec=_prec(fbs, prec)) as ctx:
        agg, di, ds = ctx.aggregate(_dev(cost), _dev(G), 0, 1.0, 10.0)
        torch.cuda.synchronize()
        fbs.fbs_sync(ctx.ctx)
    np.testing.assert_array_equal(agg.cpu().numpy(), _round16(cost, prec))


@pytest.mark.parametrize("prec", ["bf16", "f16"])
@pytest.mark.parametrize("H,W,C,D,r", [(16, 24, 3, 16, 2), (21, 45, 3, 40, 7), (9, 70, 1, 64, 4), (30, 33, 3, 100, 9),
                                       (18, 300, 3, 256, 9), (11, 270, 1, 245, 5)])
def test_tc_aggregation_within_rounding_bound(fbs, oracle_mod, prec, H, W, C, D, r):
    rng = np.random.default_rng(7 * H + W)
    L = rng.integers(0, 256, size=(H, W, C)).astype(np.uint8)
    R = np.roll(L, -3, axis=1)
    with fbs.Context(0, prec=_prec(fbs, prec)) as ctx:
        dl, dr = _dev(L), _dev(R)
        cost = ctx.cost_volume(dl, dr, D)
        agg, di, ds = ctx.aggregate(cost, dl, r, float(r), 12.0)
        di2, ds2 = ctx.compute_disparity(dl, dr, D, r, float(r), 12.0)
        torch.cuda.synchronize()
        fbs.fbs_sync(ctx.ctx)
    ref_di, ref_ds, ref_agg = oracle_mod.fbs(L, R, D, r, float(r), 12.0, want_agg=True)
    err = np.abs(agg.cpu().numpy() - ref_agg).max()
    tol = 3 * U[prec] * 2.0 + 1e-5
    assert err <= tol, f"max |dAgg| {err:.3e} > {tol:.3e}"
    # integer winners agree except where the oracle's two best are within 2*tol,
    # subpixel disparities within the rounding bound propagated through Eq. (10)
    di = di.cpu().numpy()
    ties = near_tie_mask(ref_agg, 2 * tol)
    assert np.all((di == ref_di) | ties)
    stats = check_disparities(di, ds.cpu().numpy(), ref_agg, ref_di, ref_ds, 2.0, tol=tol)
    print(f"{prec} {W}x{H} D={D} r={r}: max |dAgg| {err:.2e} (bound {tol:.2e}), {stats}")
    # the production entry point (16-bit cost built directly) agrees with the
    # debug route (FP32 cost rounded by the conversion kernel): same rounding
    assert np.array_equal(di, di2.cpu().numpy())
    np.testing.assert_allclose(ds.cpu().numpy(), ds2.cpu().numpy(), atol=1e-6)


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_tc_full_size_bench_workload_bad_pixels(fbs, oracle_mod, prec):
    """640x480 RGB, D=64, radius 7 (the benchmark workload): aggregated costs
    of 400 sampled pixels within the 16-bit rounding bound of the FP64 oracle
    (the largest error is printed), their integer and subpixel disparities
    under the 16-bit rules, and extra bad pixels (> 1 px) of the 16-bit form
    over the FP32 form at most 0.5% on the sample and on the whole frame."""
    from synth import make_pair
    p = make_pair("rgb640x480_d64_r7", 0)
    dl, dr = _dev(p.left), _dev(p.right)
    out = {}
    for name, pr in [("f32", fbs.FBS_PREC_F32), (prec, _prec(fbs, prec))]:
        with fbs.Context(0, prec=pr) as ctx:
            di, ds = ctx.compute_disparity(dl, dr, p.D, p.radius, p.sigma_s, p.sigma_r, p.tau)
            torch.cuda.synchronize()
            fbs.fbs_sync(ctx.ctx)
            out[name] = (di.cpu().numpy(), ds.cpu().numpy())
    # the aggregated volume of the 16-bit form (debug route: the FP32 cost
    # rounded by the conversion kernel, the same rounding as the cost kernel)
    with fbs.Context(0, prec=_prec(fbs, prec)) as ctx:
        cost = ctx.cost_volume(dl, dr, p.D)
        agg, adi, ads = ctx.aggregate(cost, dl, p.radius, p.sigma_s, p.sigma_r)
        torch.cuda.synchronize()
        fbs.fbs_sync(ctx.ctx)
    assert np.array_equal(adi.cpu().numpy(), out[prec][0])
    rng = np.random.default_rng(1)
    ys = rng.integers(0, p.H, 400)
    xs = rng.integers(0, p.W, 400)
    ref_di, ref_ds, ref_agg = oracle_mod.fbs_points(p.left, p.right, p.D, p.radius, p.sigma_s, p.sigma_r, xs, ys)
    agg_s = agg[torch.from_numpy(ys).cuda(), torch.from_numpy(xs).cuda()].cpu().numpy()
    err = float(np.abs(agg_s - ref_agg).max())
    tol = 3 * U[prec] * 2.0 + 1e-5
    stats = check_disparities(out[prec][0][ys, xs], out[prec][1][ys, xs], ref_agg, ref_di, ref_ds, 2.0, tol=tol)
    print(f"640x480 D=64 r=7 {prec}: max |dAgg| vs FP64 oracle {err:.3e} (bound {tol:.3e}); {stats}")
    assert err <= tol
    bad32 = np.mean(np.abs(out["f32"][1][ys, xs] - ref_ds) > 1.0)
    bad16 = np.mean(np.abs(out[prec][1][ys, xs] - ref_ds) > 1.0)
    assert bad16 - bad32 <= 0.005, (bad32, bad16)
    # whole frame against the FP32 path
    whole = float(np.mean(np.abs(out[prec][1] - out["f32"][1]) > 1.0))
    print(f"640x480 D=64 r=7 {prec}: extra bad pixels over FP32 {100 * whole:.4f}%")
    assert whole <= 0.005


def test_tc_f16_1280x960_d128_r15(fbs, oracle_mod):
    """The precision-at-scale workload: 1280x960 RGB, D=128, radius 15, FP16
    operands.  Sampled aggregated costs within the FP16 rounding bound of the
    FP64 oracle; extra bad pixels (> 1 px) over the FP32 form at most 0.5%."""
    from synth import make_pair
    p = make_pair("rgb1280x960_d128_r15", 0)
    dl, dr = _dev(p.left), _dev(p.right)
    with fbs.Context(0, prec=fbs.FBS_PREC_F32) as c32:
        _, ds32 = c32.compute_disparity(dl, dr, p.D, p.radius, p.sigma_s, p.sigma_r)
        torch.cuda.synchronize()
    with fbs.Context(0, prec=fbs.FBS_PREC_F16) as c16:
        di16, ds16 = c16.compute_disparity(dl, dr, p.D, p.radius, p.sigma_s, p.sigma_r)
        cost = c16.cost_volume(dl, dr, p.D)
        agg, _, _ = c16.aggregate(cost, dl, p.radius, p.sigma_s, p.sigma_r)
        torch.cuda.synchronize()
        fbs.fbs_sync(c16.ctx)
    rng = np.random.default_rng(9)
    xs, ys = rng.integers(0, p.W, 60), rng.integers(0, p.H, 60)
    ref_di, ref_ds, ref_agg = oracle_mod.fbs_points(p.left, p.right, p.D, p.radius, p.sigma_s, p.sigma_r, xs, ys)
    agg_s = agg[torch.from_numpy(ys).cuda(), torch.from_numpy(xs).cuda()].cpu().numpy()
    err = np.abs(agg_s - ref_agg).max()
    tol = 3 * U["f16"] * 2.0 + 1e-5
    stats = check_disparities(di16.cpu().numpy()[ys, xs], ds16.cpu().numpy()[ys, xs], ref_agg, ref_di, ref_ds, 2.0,
                              tol=tol)
    print(f"1280x960 D=128 r=15 FP16: max |dAgg| vs FP64 oracle {err:.3e} (bound {tol:.3e}); {stats}")
    assert err <= tol
    bad = float(np.mean(np.abs(ds16.cpu().numpy() - ds32.cpu().numpy()) > 1.0))
    print(f"extra bad pixels over FP32: {100 * bad:.4f}%")
    assert bad <= 0.005


@pytest.mark.parametrize("prec,expect", [("f32", {"COST": 2, "AGG_F32": 1, "AGG_TC": 0}),
                                         ("bf16", {"COST": 1, "AGG_F32": 0, "AGG_TC": 1})])
def test_kernel_accounting_counts_every_launch(fbs, prec, expect):
    """fbs_profile_read reports kernels, not calls: the FP32 form launches the
    statistics pre-pass, the cost kernel and the aggregation; the 16-bit form
    one cost kernel (statistics, pad rows and guide included) and the
    tensor-core aggregation."""
    rng = np.random.default_rng(3)
    L = rng.integers(0, 256, size=(40, 72, 3)).astype(np.uint8)
    R = np.roll(L, -2, axis=1)
    p = fbs.FBS_PREC_F32 if prec == "f32" else _prec(fbs, prec)
    with fbs.Context(0, prec=p) as ctx:
        dl, dr = _dev(L), _dev(R)
        ctx.compute_disparity(dl, dr, 24, 3, 3.0, 12.0)
        torch.cuda.synchronize()
        fbs.fbs_profile(ctx.ctx, 1)
        for _ in range(3):
            ctx.compute_disparity(dl, dr, 24, 3, 3.0, 12.0)
        torch.cuda.synchronize()
        got = {k: fbs.fbs_profile_read(ctx.ctx, getattr(fbs, "FBS_KERNEL_" + k))[1] for k in expect}
        fbs.fbs_profile(ctx.ctx, 0)
        fbs.fbs_sync(ctx.ctx)
    assert got == {k: 3 * v for k, v in expect.items()}

