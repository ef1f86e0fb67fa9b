"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Small cases run the oracle on the whole frame; the full-size workload the
benchmark times is checked on sampled pixels (oracle point evaluation) and on
a row band.  Comparison rules are in tests/_compare.py.
"""

import numpy as np
import pytest

from tests._compare import check_agg, check_disparities

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fbs():
    from paper_1807_02044_gb300 import build as b
    b.build()
    import paper_1807_02044_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(fbs):
    c = fbs.Context(0)
    yield c
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rand(rng, H, W, C):
    return rng.integers(0, 256, size=(H, W, C)).astype(np.uint8)


def _full_path(fbs, ctx, L, R, D, radius, ss, sr, tau=0.0, cost_mode=0):
    """GPU: cost volume, aggregated volume and disparities through the debug
    entry points, plus the production entry point's disparities."""
    H, W, C = L.shape
    dl, dr = _dev(L), _dev(R)
    ctx.set_options(cost=cost_mode)
    cost = ctx.cost_volume(dl, dr, D, tau)
    agg, di, ds = ctx.aggregate(cost, dl, radius, ss, sr)
    di2, ds2 = ctx.compute_disparity(dl, dr, D, radius, ss, sr, tau)
    torch.cuda.synchronize()
    ctx.set_options(cost=0)
    return (cost.cpu().numpy(), agg.cpu().numpy(), di.cpu().numpy(), ds.cpu().numpy(),
            di2.cpu().numpy(), ds2.cpu().numpy())


CASES = [
    # H, W, C, D, radius, sigma_s, sigma_r
    (16, 24, 1, 8, 2, 2.0, 10.0),
    (13, 37, 3, 19, 3, 3.0, 12.0),       # ragged tile edges, D not a multiple of 4
    (9, 70, 3, 40, 4, 4.0, 12.0),        # two disparity chunks, second one partial
    (21, 33, 1, 100, 1, 1.5, 8.0),       # D > W, three chunks
    (11, 45, 3, 16, 0, 1.0, 12.0),       # radius 0
    (40, 18, 3, 12, 9, 6.0, 15.0),       # window wider than the tile
    (1, 1, 1, 1, 0, 1.0, 1.0),           # single pixel, single disparity
    (1, 50, 3, 7, 5, 5.0, 12.0),         # single row
    (30, 1, 1, 3, 2, 2.0, 10.0),         # single column
]


@pytest.mark.parametrize("H,W,C,D,radius,ss,sr", CASES)
def test_path_matches_oracle_small(fbs, ctx, oracle_mod, H, W, C, D, radius, ss, sr):
    rng = np.random.default_rng(H * 1000 + W * 10 + C)
    L = _rand(rng, H, W, C)
    R = np.roll(L, -min(3, W - 1), axis=1)
    R = np.clip(R.astype(np.int32) + rng.integers(-6, 7, R.shape), 0, 255).astype(np.uint8)
    cost, agg, di, ds, di2, ds2 = _full_path(fbs, ctx, L, R, D, radius, ss, sr)
    ref_cost = oracle_mod.cost_volume(L, R, D)
    check_agg(cost, ref_cost, 2.0)          # cost is within 1e-5 of its range too
    ref_di, ref_ds, ref_agg = oracle_mod.fbs(L, R, D, radius, ss, sr, want_agg=True)
    err = check_agg(agg, ref_agg, 2.0)
    check_disparities(di, ds, ref_agg, ref_di, ref_ds, 2.0, err)
    # the production entry point runs the same arithmetic
    assert np.array_equal(di, di2)
    assert np.array_equal(ds, ds2)


@pytest.mark.parametrize("tau", [20.0, 5.0])
def test_tad_mode_matches_oracle(fbs, ctx, oracle_mod, tau):
    rng = np.random.default_rng(77)
    L = _rand(rng, 12, 40, 3)
    R = np.roll(L, -4, axis=1)
    cost, agg, di, ds, di2, ds2 = _full_path(fbs, ctx, L, R, 12, 3, 3.0, 12.0, tau=tau, cost_mode=1)
    ref_cost = oracle_mod.cost_volume(L, R, 12, oracle_mod.COST_TAD, tau)
    check_agg(cost, ref_cost, tau)
    ref_di, ref_ds, ref_agg = oracle_mod.fbs(L, R, 12, 3, 3.0, 12.0, tau=tau, mode=oracle_mod.COST_TAD,
                                             want_agg=True)
    err = check_agg(agg, ref_agg, tau)
    check_disparities(di, ds, ref_agg, ref_di, ref_ds, tau, err)


def test_aggregation_alone_on_oracle_cost(fbs, ctx, oracle_mod):
    """Isolates steps 2-4: the oracle's cost volume (rounded to FP32) in, the
    oracle's aggregation of the same FP32 values as the reference."""
    rng = np.random.default_rng(5)
    H, W, C, D, r = 20, 44, 3, 24, 5
    G = _rand(rng, H, W, C)
    cost32 = rng.random((H, W, D)).astype(np.float32) * 2
    agg, di, ds = ctx.aggregate(_dev(cost32), _dev(G), r, 4.0, 12.0)
    torch.cuda.synchronize()
    ref_agg = oracle_mod.aggregate(cost32.astype(np.float64), G, r, 4.0, 12.0)
    err = check_agg(agg.cpu().numpy(), ref_agg, 2.0)
    ref_di, ref_ds = oracle_mod.wta_subpixel(ref_agg)
    check_disparities(di.cpu().numpy(), ds.cpu().numpy(), ref_agg, ref_di, ref_ds, 2.0, err)


def test_subpixel_vertex_of_exact_quadratic_through_radius_zero(fbs, ctx):
    """Agg(d) = alpha (d - d_v)^2 + beta fed through the aggregation with
    radius 0 (Agg = C) returns d_v (Eq. (10) is exact on a parabola)."""
    H, W, D = 3, 40, 32
    rng = np.random.default_rng(1)
    dv = rng.uniform(1.0, D - 2.0, size=(H, W))
    alpha = rng.uniform(0.001, 0.05, size=(H, W))
    d = np.arange(D)
    cost = (alpha[..., None] * (d - dv[..., None]) ** 2 + 0.1).astype(np.float32)
    G = _rand(rng, H, W, 3)
    _, di, ds = ctx.aggregate(_dev(cost), _dev(G), 0, 1.0, 10.0, want_agg=False)
    torch.cuda.synchronize()
    assert np.abs(ds.cpu().numpy() - dv).max() < 1e-3


def test_shifted_texture_recovers_disparity_on_gpu(fbs, ctx):
    from synth import shifted_texture_pair
    d0, r = 11, 4
    L, R = shifted_texture_pair(40, 96, 3, d0, seed=3)
    di, ds = ctx.compute_disparity(_dev(L), _dev(R), 32, r, 4.0, 12.0)
    torch.cuda.synchronize()
    di = di.cpu().numpy()
    assert np.all(di[:, d0 + 1 + r: 96 - 2 - r] == d0)


def test_constant_images_give_flat_costs(fbs, ctx):
    L = np.full((8, 20, 3), 50, np.uint8)
    cost = ctx.cost_volume(_dev(L), _dev(L), 6).cpu().numpy()
    for d in range(6):
        assert np.all(cost[:, d:, d] == 1.0)
        assert np.all(cost[:, :d, d] == 2.0)


def test_host_entry_point_matches_device_path(fbs, ctx):
    rng = np.random.default_rng(9)
    L = _rand(rng, 33, 57, 3)
    R = np.roll(L, -5, axis=1)
    di, ds = ctx.compute_disparity(_dev(L), _dev(R), 20, 3, 3.0, 12.0)
    torch.cuda.synchronize()
    hi = np.empty((33, 57), np.int32)
    hs = np.empty((33, 57), np.float32)
    fbs.fbs_compute_disparity_host(ctx.ctx, L, R, 33, 57, 3, 20, 3, 3.0, 12.0, 0.0, hi, hs)
    assert np.array_equal(hi, di.cpu().numpy())
    assert np.array_equal(hs, ds.cpu().numpy())


@pytest.mark.parametrize("prec", ["bf16", "f16"])
@pytest.mark.parametrize("H,W,D,r,mode", [(33, 57, 20, 3, 0), (480, 640, 64, 7, 0), (61, 90, 40, 15, 0),
                                          (7, 30, 12, 2, 0), (100, 77, 24, 4, 1)])
def test_host_entry_point_tensor_cores(fbs, prec, H, W, D, r, mode):
    """The tensor-core form of the host-buffer call (upload, the path,
    download) returns exactly what the device-buffer call returns, with
    pageable and with pinned host buffers, also with one output omitted and on
    new contents of the same buffers."""
    rng = np.random.default_rng(H * W + D)
    L = _rand(rng, H, W, 3)
    R = np.roll(L, -5, axis=1)
    p = fbs.FBS_PREC_BF16 if prec == "bf16" else fbs.FBS_PREC_F16
    with fbs.Context(0, cost=mode, prec=p) as c16:
        di, ds = c16.compute_disparity(_dev(L), _dev(R), D, r, float(r), 12.0, 20.0)
        torch.cuda.synchronize()
        di, ds = di.cpu().numpy(), ds.cpu().numpy()
        # pageable numpy buffers
        hi = np.full((H, W), -9, np.int32)
        hs = np.full((H, W), -9, np.float32)
        fbs.fbs_compute_disparity_host(c16.ctx, L, R, H, W, 3, D, r, float(r), 12.0, 20.0, hi, hs)
        assert np.array_equal(hi, di)
        assert np.array_equal(hs.view(np.uint32), ds.view(np.uint32))
        # pinned buffers, twice
        pl = torch.from_numpy(L).pin_memory()
        pr = torch.from_numpy(R).pin_memory()
        pi = torch.full((H, W), -9, dtype=torch.int32).pin_memory()
        ps = torch.full((H, W), -9.0).pin_memory()
        for _ in range(2):
            pi.fill_(-9)
            ps.fill_(-9.0)
            fbs.fbs_compute_disparity_host(c16.ctx, pl, pr, H, W, 3, D, r, float(r), 12.0, 20.0, pi, ps)
            assert np.array_equal(pi.numpy(), di)
            assert np.array_equal(ps.numpy().view(np.uint32), ds.view(np.uint32))
        ps2 = torch.full((H, W), -9.0).pin_memory()
        fbs.fbs_compute_disparity_host(c16.ctx, pl, pr, H, W, 3, D, r, float(r), 12.0, 20.0, None, ps2)
        assert np.array_equal(ps2.numpy().view(np.uint32), ds.view(np.uint32))
        # new contents of the same pinned buffers
        L2 = L[::-1].copy()
        R2 = R[::-1].copy()
        pl.copy_(torch.from_numpy(L2))
        pr.copy_(torch.from_numpy(R2))
        fbs.fbs_compute_disparity_host(c16.ctx, pl, pr, H, W, 3, D, r, float(r), 12.0, 20.0, pi, ps)
        d2i, d2s = c16.compute_disparity(_dev(L2), _dev(R2), D, r, float(r), 12.0, 20.0)
        torch.cuda.synchronize()
        assert np.array_equal(pi.numpy(), d2i.cpu().numpy())
        assert np.array_equal(ps.numpy().view(np.uint32), d2s.cpu().numpy().view(np.uint32))
        fbs.fbs_sync(c16.ctx)


def test_invalid_arguments_are_rejected_before_launch(fbs, ctx):
    L = _dev(np.zeros((4, 4, 3), np.uint8))
    out = torch.empty((4, 4), dtype=torch.int32, device="cuda")
    bad = [
        dict(H=0), dict(W=-1), dict(C=2), dict(D=0), dict(D=2000), dict(radius=-1), dict(radius=32),
        dict(sigma_s=0.0), dict(sigma_r=-1.0), dict(sigma_s=float("nan")),
    ]
    for b in bad:
        args = dict(H=4, W=4, C=3, D=4, radius=1, sigma_s=1.0, sigma_r=1.0)
        args.update(b)
        with pytest.raises(fbs.FBSError) as ei:
            fbs.fbs_compute_disparity(ctx.ctx, L, L, args["H"], args["W"], args["C"], args["D"], args["radius"],
                                      args["sigma_s"], args["sigma_r"], 0.0, out, None)
        assert ei.value.status == fbs.FBS_ERR_INVALID_ARG
    with pytest.raises(fbs.FBSError):
        fbs.fbs_compute_disparity(ctx.ctx, None, L, 4, 4, 3, 4, 1, 1.0, 1.0, 0.0, out, None)
    with pytest.raises(fbs.FBSError):
        fbs.fbs_compute_disparity(ctx.ctx, L, L, 4, 4, 3, 4, 1, 1.0, 1.0, 0.0, None, None)
    # TAD mode needs tau >= 0
    ctx.set_options(cost=1)
    try:
        with pytest.raises(fbs.FBSError):
            fbs.fbs_compute_disparity(ctx.ctx, L, L, 4, 4, 3, 4, 1, 1.0, 1.0, -1.0, out, None)
    finally:
        ctx.set_options(cost=0)
    fbs.fbs_sync(ctx.ctx)


def test_workspace_cap_gives_oom_status(fbs):
    c = fbs.Context(0, workspace_cap=1024)
    try:
        L = _dev(np.zeros((64, 64, 1), np.uint8))
        with pytest.raises(fbs.FBSError) as ei:
            c.compute_disparity(L, L, 16, 2, 2.0, 10.0)
        assert ei.value.status == fbs.FBS_ERR_OOM
    finally:
        c.close()


# ---------------------------------------------------------------------------
# The benchmark's workload at full size (640x480 RGB, D=64, radius 7)
# ---------------------------------------------------------------------------
def test_full_size_bench_workload_sampled(fbs, ctx, oracle_mod):
    from synth import make_pair
    p = make_pair("rgb640x480_d64_r7", 0)
    dl, dr = _dev(p.left), _dev(p.right)
    di, ds = ctx.compute_disparity(dl, dr, p.D, p.radius, p.sigma_s, p.sigma_r, p.tau)
    cost = ctx.cost_volume(dl, dr, p.D)
    agg, _, _ = ctx.aggregate(cost, dl, p.radius, p.sigma_s, p.sigma_r)
    torch.cuda.synchronize()
    di, ds, agg = di.cpu().numpy(), ds.cpu().numpy(), agg.cpu().numpy()
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.integers(0, p.W, 150), [0, p.W - 1, 0, p.W - 1, 7, 320]])
    ys = np.concatenate([rng.integers(0, p.H, 150), [0, 0, p.H - 1, p.H - 1, 239, 3]])
    ref_di, ref_ds, ref_agg = oracle_mod.fbs_points(p.left, p.right, p.D, p.radius, p.sigma_s, p.sigma_r, xs, ys)
    err = check_agg(agg[ys, xs], ref_agg, 2.0)
    check_disparities(di[ys, xs], ds[ys, xs], ref_agg, ref_di, ref_ds, 2.0, err)
    # a row band of the same frame, oracle on whole rows
    y0, y1 = 232, 236
    bi, bs, bagg = oracle_mod.fbs(p.left, p.right, p.D, p.radius, p.sigma_s, p.sigma_r, rows=(y0, y1),
                                  want_agg=True)
    err = check_agg(agg[y0:y1], bagg, 2.0)
    stats = check_disparities(di[y0:y1], ds[y0:y1], bagg, bi, bs, 2.0, err)
    assert stats["near_ties"] < 0.01 * stats["pixels"]


# ---------------------------------------------------------------------------
# The other stated workloads
# ---------------------------------------------------------------------------
def test_gray160x120_whole_frame(fbs, ctx, oracle_mod):
    """160x120 grey, D=16, radius 4 (9x9), sigma_s 4, sigma_r 10: every pixel
    against the oracle."""
    from synth import make_pair
    p = make_pair("gray160x120_d16_r4", 0)
    dl, dr = _dev(p.left), _dev(p.right)
    cost = ctx.cost_volume(dl, dr, p.D)
    agg, di, ds = ctx.aggregate(cost, dl, p.radius, p.sigma_s, p.sigma_r)
    di2, ds2 = ctx.compute_disparity(dl, dr, p.D, p.radius, p.sigma_s, p.sigma_r)
    torch.cuda.synchronize()
    ref_di, ref_ds, ref_agg = oracle_mod.fbs(p.left, p.right, p.D, p.radius, p.sigma_s, p.sigma_r, want_agg=True)
    err = check_agg(agg.cpu().numpy(), ref_agg, 2.0)
    check_disparities(di2.cpu().numpy(), ds2.cpu().numpy(), ref_agg, ref_di, ref_ds, 2.0, err)


def test_full_size_1280x960_sampled(fbs, ctx, oracle_mod):
    """1280x960 RGB, D=128, radius 15 (31x31): 120 sampled pixels against the
    oracle's point evaluation."""
    from synth import make_pair
    p = make_pair("rgb1280x960_d128_r15", 0)
    dl, dr = _dev(p.left), _dev(p.right)
    cost = ctx.cost_volume(dl, dr, p.D)
    agg, di, ds = ctx.aggregate(cost, dl, p.radius, p.sigma_s, p.sigma_r)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    xs = np.concatenate([rng.integers(0, p.W, 116), [0, p.W - 1, 0, p.W - 1]])
    ys = np.concatenate([rng.integers(0, p.H, 116), [0, 0, p.H - 1, p.H - 1]])
    ref_di, ref_ds, ref_agg = oracle_mod.fbs_points(p.left, p.right, p.D, p.radius, p.sigma_s, p.sigma_r, xs, ys)
    agg_s = agg[torch.from_numpy(ys).cuda(), torch.from_numpy(xs).cuda()].cpu().numpy()
    err = check_agg(agg_s, ref_agg, 2.0)
    check_disparities(di.cpu().numpy()[ys, xs], ds.cpu().numpy()[ys, xs], ref_agg, ref_di, ref_ds, 2.0, err)
