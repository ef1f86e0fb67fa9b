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
// address.  The first call on each device (with that device current) asks the
// runtime for the array's device address with cudaGetSymbolAddress, checks the
// result, and caches it; the kernels receive that address.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "fbs_internal.cuh"

namespace {

constexpr size_t kScratchFloats = FBS_NOALLOC_MAX_COST_BYTES / sizeof(float);

// Shared by every call on a device; holds the last call's statistics and cost volume.
static __device__ __align__(256) float g_noalloc_cost[kScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
float* g_scratch_addr[kMaxDevices] = {};

// Device address of g_noalloc_cost on `dev` (which must be current).
cudaError_t scratch_address(int dev, float** out)
{
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_cost);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<float*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

struct CurrentDevice {
    int prev = -1;
    bool ok = false;
    explicit CurrentDevice(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
    }
    ~CurrentDevice()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" fbs_status fbs_compute_disparity_noalloc(fbs_ctx* ctx, const uint8_t* left, const uint8_t* right,
                                                    int H, int W, int C, int D, int radius, float sigma_s,
                                                    float sigma_r, float tau, int32_t* disp_int,
                                                    float* disp_subpix, void* cuda_stream)
{
    if (!ctx) return FBS_ERR_INVALID_ARG;
    fbs::ctx_error(ctx, FBS_OK, "");
    fbs_status s = fbs::check_path_args(ctx, left, right, H, W, C, D, radius, sigma_s, sigma_r, tau, disp_int,
                                        disp_subpix);
    if (s != FBS_OK) return s;
    if (fbs::ctx_precision(ctx) != FBS_PREC_F32)
        return fbs::ctx_error(ctx, FBS_ERR_UNSUPPORTED, "fbs_compute_disparity_noalloc serves FP32 precision only");
    const int ld = fbs::padded_ld(D);
    const size_t stats = fbs::cost_scratch_bytes(H, W);
    const size_t need = stats + sizeof(float) * (size_t)H * W * ld;
    if (need > FBS_NOALLOC_MAX_COST_BYTES) {
        std::string msg = "fbs_compute_disparity_noalloc: block statistics plus cost volume need " +
                          std::to_string(need) + " bytes, which exceeds the static scratch of " +
                          std::to_string((size_t)FBS_NOALLOC_MAX_COST_BYTES) + " bytes";
        return fbs::ctx_error(ctx, FBS_ERR_INVALID_ARG, msg.c_str());
    }
    const int dev = fbs::ctx_device(ctx);
    if (dev < 0 || dev >= kMaxDevices) return fbs::ctx_error(ctx, FBS_ERR_UNSUPPORTED, "device ordinal too large");
    CurrentDevice guard(dev);
    if (!guard.ok) return fbs::ctx_error(ctx, FBS_ERR_CUDA, "cannot select the context's device");
    float* scratch = nullptr;
    cudaError_t e = scratch_address(dev, &scratch);
    if (e != cudaSuccess) {
        std::string msg = std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e);
        return fbs::ctx_error(ctx, FBS_ERR_CUDA, msg.c_str());
    }
    cudaStream_t st = fbs::ctx_stream(ctx, cuda_stream);
    // [block statistics | cost volume]; every element a kernel reads is written
    // earlier in the same call (padding lanes included), so nothing in the
    // array needs clearing.
    const fbs::CostScratch sc = fbs::carve_cost_scratch(scratch, H, W);
    float* cost = (float*)((uint8_t*)scratch + stats);
    long long k0 = fbs::launch_count();
    e = fbs::launch_cost_build(sc, left, right, H, W, C, D, ld, fbs::ctx_cost_mode(ctx), tau, cost, st);
    fbs::ctx_count_launch(ctx, FBS_KERNEL_COST, fbs::launch_count() - k0);
    if (e != cudaSuccess) {
        std::string msg = std::string("cost build launch: ") + cudaGetErrorString(e);
        return fbs::ctx_error(ctx, FBS_ERR_CUDA, msg.c_str());
    }
    k0 = fbs::launch_count();
    e = fbs::launch_aggregate_f32(cost, ld, left, H, W, C, D, radius, sigma_s, sigma_r, nullptr, disp_int,
                                  disp_subpix, st);
    fbs::ctx_count_launch(ctx, FBS_KERNEL_AGG_F32, fbs::launch_count() - k0);
    if (e != cudaSuccess) {
        std::string msg = std::string("aggregation launch: ") + cudaGetErrorString(e);
        return fbs::ctx_error(ctx, FBS_ERR_CUDA, msg.c_str());
    }
    return FBS_OK;
}
