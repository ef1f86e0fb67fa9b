// Both disparity maps and the left-right consistency check: each matching
// cost is computed once and stored in the left volume at (u, v, d) and in the
// right volume at (u - d, v, d) (Sec. II-A, Sec. III); each volume is
// aggregated with its own image as guide (Sec. II-B), WTA and Eq. (10) give
// both maps, and the LRC check of Eq. (9) removes the left disparities the
// right map does not confirm.
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
