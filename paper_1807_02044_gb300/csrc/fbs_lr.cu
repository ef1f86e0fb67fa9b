// Both disparity maps and the left-right consistency check (Sec. II-A,
// Sec. III, Eq. (9)).  FP32: each matching cost is computed once and stored in
// the left volume at (u, v, d) and in the right volume at (u - d, v, d); each
// volume is aggregated with its own image as guide (Sec. II-B), WTA and
// Eq. (10) give both maps.  BF16 / FP16: the tensor-core path runs on the pair
// and on its mirrored, swapped copy (whose left view is the mirrored right
// view).  The LRC check removes the left disparities the right map does not
// confirm.
#include <cuda_runtime.h>

#include "fbs_context.cuh"

using namespace fbs_detail;

namespace {

// Eq. (9): keep d = dl(u, v) only when u - d >= 0 and dr(u - d, v) == d; a
// rejected pixel gets -1 in both left outputs.
__global__ void lrc_kernel(const int32_t* __restrict__ dl, const int32_t* __restrict__ dr, int H, int W,
                           int32_t* __restrict__ out_int, float* __restrict__ out_sub)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y;
    if (u >= W) return;
    const size_t p = (size_t)v * W + u;
    const int d = dl[p];
    const bool ok = u - d >= 0 && dr[p - d] == d;
    if (!ok) {
        if (out_int) out_int[p] = -1;
        if (out_sub) out_sub[p] = -1.f;
    }
}

// Horizontal mirror of both images with the views swapped: out_l = mirror(R),
// out_r = mirror(L).  The right view of (L, R) is the mirrored left view of
// (out_l, out_r): the cost of right pixel u at d, NCC(R block at u, L block at
// u + d), is the cost of pixel W-1-u of out_l against out_r at W-1-u-d, with the
// same clamped blocks, and u + d >= W becomes W-1-u - d < 0.
__global__ void mirror_swap_kernel(const uint8_t* __restrict__ L, const uint8_t* __restrict__ R, int H, int W, int C,
                                   uint8_t* __restrict__ out_l, uint8_t* __restrict__ out_r)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W) return;
    const uint8_t* src = blockIdx.z == 0 ? R : L;
    uint8_t* dst = blockIdx.z == 0 ? out_l : out_r;
    const size_t i = ((size_t)y * W + x) * C, j = ((size_t)y * W + (W - 1 - x)) * C;
    for (int c = 0; c < C; ++c) dst[i + c] = src[j + c];
}

// Right-view maps back from the mirrored frame: right pixel u is mirrored pixel W-1-u.
__global__ void unmirror_maps_kernel(const int32_t* __restrict__ mi, const float* __restrict__ ms, int H, int W,
                                     int32_t* __restrict__ di, float* __restrict__ ds)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W) return;
    const size_t o = (size_t)y * W + x, m = (size_t)y * W + (W - 1 - x);
    if (di) di[o] = mi[m];
    if (ds) ds[o] = ms[m];
}

// BF16 / FP16 contexts: both views on the tensor cores.  The left view is
// fbs_compute_disparity's tensor-core path; the right view is the same path
// on the mirrored, swapped pair, mirrored back.
fbs_status lr_tensor_cores(fbs_ctx* ctx, const uint8_t* left, const uint8_t* right, int H, int W, int C, int D,
                           int radius, float sigma_s, float sigma_r, float tau, int32_t* disp_int,
                           float* disp_subpix, int32_t* disp_int_right, float* disp_subpix_right, int lrc,
                           cudaStream_t st)
{
    if (!fbs::tc_supported(D, radius))
        return fail(ctx, FBS_ERR_UNSUPPORTED,
                    "tensor-core aggregation supports D <= 256 and radius <= 24 (got D=%d, radius=%d)", D, radius);
    const size_t img = ((size_t)H * W * C + 255) & ~(size_t)255;
    const size_t map = ((size_t)H * W * 4 + 255) & ~(size_t)255;
    // [mirrored left | mirrored right | mirrored-frame int map | float map | left int map | right int map]
    fbs_status s = ensure(ctx, &ctx->aux, &ctx->aux_bytes, 2 * img + 4 * map, "mirrored views");
    if (s != FBS_OK) return s;
    uint8_t* base = (uint8_t*)ctx->aux;
    uint8_t* ml = base;
    uint8_t* mr = base + img;
    int32_t* mi = (int32_t*)(base + 2 * img);
    float* ms = (float*)(base + 2 * img + map);
    int32_t* dl = disp_int ? disp_int : (int32_t*)(base + 2 * img + 2 * map);
    int32_t* dr = disp_int_right ? disp_int_right : (int32_t*)(base + 2 * img + 3 * map);
    const bool want_right = lrc || disp_int_right || disp_subpix_right;
    s = fbs::run_path_tc(ctx, left, right, H, W, C, D, radius, sigma_s, sigma_r, tau, dl, disp_subpix, st);
    if (s != FBS_OK || !want_right) return s;
    const dim3 grid((W + 255) / 256, H);
    cudaError_t e;
    {
        LaunchScope ls(ctx, FBS_KERNEL_OTHER, st);
        fbs::note_launch();
        mirror_swap_kernel<<<dim3(grid.x, H, 2), 256, 0, st>>>(left, right, H, W, C, ml, mr);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mirror launch");
    s = fbs::run_path_tc(ctx, ml, mr, H, W, C, D, radius, sigma_s, sigma_r, tau, mi, ms, st);
    if (s != FBS_OK) return s;
    {
        LaunchScope ls(ctx, FBS_KERNEL_OTHER, st);
        fbs::note_launch();
        unmirror_maps_kernel<<<grid, 256, 0, st>>>(mi, ms, H, W, dr, disp_subpix_right);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "unmirror launch");
    if (lrc) {
        LaunchScope ls(ctx, FBS_KERNEL_OTHER, st);
        fbs::note_launch();
        lrc_kernel<<<grid, 256, 0, st>>>(dl, dr, H, W, disp_int, disp_subpix);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "LRC launch");
    }
    return FBS_OK;
}

}  // namespace

extern "C" fbs_status fbs_compute_disparity_lr(fbs_ctx* ctx, const uint8_t* left, const uint8_t* right, int H,
                                               int W, int C, int D, int radius, float sigma_s, float sigma_r,
                                               float tau, int32_t* disp_int, float* disp_subpix,
                                               int32_t* disp_int_right, float* disp_subpix_right, int lrc,
                                               void* cuda_stream)
{
    if (!ctx) return FBS_ERR_INVALID_ARG;
    fbs_status s = fbs::check_path_args(ctx, left, right, H, W, C, D, radius, sigma_s, sigma_r, tau, disp_int,
                                        disp_subpix);
    if (s != FBS_OK) return s;
    DeviceGuard g(ctx->device);
    cudaStream_t st = pick_stream(ctx, cuda_stream);
    if (ctx->opt.prec != FBS_PREC_F32)
        return lr_tensor_cores(ctx, left, right, H, W, C, D, radius, sigma_s, sigma_r, tau, disp_int, disp_subpix,
                               disp_int_right, disp_subpix_right, lrc, st);
    const int ld = fbs::padded_ld(D);
    const size_t stats = fbs::cost_scratch_bytes(H, W);
    const size_t vol = ((sizeof(float) * (size_t)H * W * ld) + 255) & ~(size_t)255;
    const size_t imap = ((sizeof(int32_t) * (size_t)H * W) + 255) & ~(size_t)255;
    s = ensure(ctx, &ctx->ws, &ctx->ws_bytes, stats + 2 * vol + 2 * imap, "cost volumes of both views");
    if (s != FBS_OK) return s;
    uint8_t* base = (uint8_t*)ctx->ws;
    const fbs::CostScratch sc = fbs::carve_cost_scratch(base, H, W);
    float* cost_l = (float*)(base + stats);
    float* cost_r = (float*)(base + stats + vol);
    // integer maps the check needs when the caller does not ask for them
    int32_t* dl = disp_int ? disp_int : (int32_t*)(base + stats + 2 * vol);
    int32_t* dr = disp_int_right ? disp_int_right : (int32_t*)(base + stats + 2 * vol + imap);
    const bool want_right = lrc || disp_int_right || disp_subpix_right;
    cudaError_t e;
    {
        LaunchScope ls(ctx, FBS_KERNEL_COST, st);
        e = fbs::launch_cost_build_lr(sc, left, right, H, W, C, D, ld, ctx->opt.cost, tau, cost_l, cost_r, st);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cost build (both views) launch");
    {
        LaunchScope ls(ctx, FBS_KERNEL_AGG_F32, st);
        e = fbs::launch_aggregate_f32(cost_l, ld, left, H, W, C, D, radius, sigma_s, sigma_r, nullptr, dl,
                                      disp_subpix, st);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "left aggregation launch");
    if (want_right) {
        LaunchScope ls(ctx, FBS_KERNEL_AGG_F32, st);
        e = fbs::launch_aggregate_f32(cost_r, ld, right, H, W, C, D, radius, sigma_s, sigma_r, nullptr, dr,
                                      disp_subpix_right, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "right aggregation launch");
    }
    if (lrc) {
        LaunchScope ls(ctx, FBS_KERNEL_OTHER, st);
        fbs::note_launch();
        lrc_kernel<<<dim3((W + 255) / 256, H), 256, 0, st>>>(dl, dr, H, W, disp_int, disp_subpix);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "LRC launch");
    }
    return FBS_OK;
}
