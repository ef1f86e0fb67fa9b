// fbs_compute_disparity_noalloc: the whole path with no device allocation.
//
// Some callers cannot call cudaMalloc once they are running -- for example a
// plugin inside a host application that owns all device memory through its own
// allocator, or a real-time loop whose memory budget is fixed at start-up and
// which may not take the allocation (or the synchronisation that cudaMalloc
// and cudaFree can imply) in the middle of processing.  This entry point gives
// them the same result as fbs_compute_disparity without touching the
// context's grow-on-demand scratch: the per-pixel block statistics and the
// cost volume live in one file-scope device array of fixed size, part of the
// library's device code.
//
// The array's name is a host-side stand-in in host code, not a device
// address.  Every call asks the runtime for the array's address in the CUDA
// context current on the calling thread once the context's device has been
// selected (cudaGetSymbolAddress: a host-side lookup that allocates nothing),
// and the kernels launched in that same CUDA context receive it.  Nothing is
// cached, so a caller that switches between the primary context and its own
// driver-API context on the same device gets each context's own copy.
#include <cuda_runtime.h>

#include "fbs_context.cuh"

using namespace fbs_detail;

namespace {

constexpr size_t kScratchFloats = FBS_NOALLOC_MAX_COST_BYTES / sizeof(float);

// Shared by every call in a CUDA context; holds the last call's statistics and cost volume.
static __device__ __align__(256) float g_noalloc_cost[kScratchFloats];

}  // namespace

extern "C" fbs_status fbs_compute_disparity_noalloc(fbs_ctx* ctx, const uint8_t* left, const uint8_t* right,
                                                    int H, int W, int C, int D, int radius, float sigma_s,
                                                    float sigma_r, float tau, int32_t* disp_int,
                                                    float* disp_subpix, void* cuda_stream)
{
    if (!ctx) return FBS_ERR_INVALID_ARG;
    ctx->err.clear();
    fbs_status s = fbs::check_path_args(ctx, left, right, H, W, C, D, radius, sigma_s, sigma_r, tau, disp_int,
                                        disp_subpix);
    if (s != FBS_OK) return s;
    if (ctx->opt.prec != FBS_PREC_F32)
        return fail(ctx, FBS_ERR_UNSUPPORTED, "fbs_compute_disparity_noalloc serves FP32 precision only");
    const int ld = fbs::padded_ld(D);
    const size_t stats = fbs::cost_scratch_bytes(H, W);
    const size_t need = stats + sizeof(float) * (size_t)H * W * ld;
    if (need > FBS_NOALLOC_MAX_COST_BYTES)
        return fail(ctx, FBS_ERR_INVALID_ARG,
                    "fbs_compute_disparity_noalloc: block statistics plus cost volume need %zu bytes, which exceeds "
                    "the static scratch of %zu bytes",
                    need, (size_t)FBS_NOALLOC_MAX_COST_BYTES);
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return fail(ctx, FBS_ERR_CUDA, "cannot select the context's device");
    fbs_status inj = take_injected_failure(ctx);
    if (inj != FBS_OK) return inj;
    void* scratch = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&scratch, g_noalloc_cost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetSymbolAddress of the static scratch");
    cudaStream_t st = pick_stream(ctx, cuda_stream);
    // [block statistics | cost volume]; every element a kernel reads is written
    // earlier in the same call (padding lanes included), so nothing in the
    // array needs clearing.
    const fbs::CostScratch sc = fbs::carve_cost_scratch(scratch, H, W);
    float* cost = (float*)((uint8_t*)scratch + stats);
    {
        LaunchScope ls(ctx, FBS_KERNEL_COST, st);
        e = fbs::launch_cost_build(sc, left, right, H, W, C, D, ld, ctx->opt.cost, tau, cost, st);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cost build launch");
    {
        LaunchScope ls(ctx, FBS_KERNEL_AGG_F32, st);
        e = fbs::launch_aggregate_f32(cost, ld, left, H, W, C, D, radius, sigma_s, sigma_r, nullptr, disp_int,
                                      disp_subpix, st);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "aggregation launch");
    return FBS_OK;
}
