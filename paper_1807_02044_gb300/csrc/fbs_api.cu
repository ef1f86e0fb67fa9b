// C ABI of libfbs: contexts, argument validation, scratch management and the
// dispatch of the fast-bilateral-stereo kernels.  See include/fbs.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>


#include "fbs_context.cuh"

using namespace fbs_detail;

namespace fbs {

// Tensor-core form: 16-bit x-blocked cost volume, tcgen05 aggregation.
fbs_status run_path_tc(fbs_ctx* ctx, const uint8_t* left, const uint8_t* right, int H, int W, int C, int D,
                       int radius, float sigma_s, float sigma_r, float tau, int32_t* disp_int, float* disp_subpix,
                       cudaStream_t st)
{
    if (!fbs::tc_supported(D, radius))
        return fail(ctx, FBS_ERR_UNSUPPORTED, "tensor-core aggregation supports D <= 256 and radius <= 24 (got D=%d, radius=%d)",
                    D, radius);
    fbs_status inj = take_injected_failure(ctx);
    if (inj != FBS_OK) return inj;
    const bool bf16 = ctx->opt.prec == FBS_PREC_BF16;
    // scratch: [packed guide | 16-bit x-blocked volume]; the cost kernel writes both
    const size_t rgbx = fbs::rgbx_bytes(H, W);
    const size_t need = rgbx + fbs::xblock16_bytes(H, W, D);
    fbs_status s = ensure(ctx, &ctx->ws, &ctx->ws_bytes, need, "cost volume");
    if (s != FBS_OK) return s;
    fbs::CostScratch sc{};
    sc.rgbx = (uint2*)ctx->ws;
    void* cost = (uint8_t*)ctx->ws + rgbx;
    cudaError_t e;
    {
        LaunchScope ls(ctx, FBS_KERNEL_COST, st);
        e = fbs::launch_cost_build_xblock16(sc, left, right, H, W, C, D, ctx->opt.cost, tau, bf16, cost, st);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cost build launch");
    {
        LaunchScope ls(ctx, FBS_KERNEL_AGG_TC, st);
        e = fbs::launch_aggregate_tc(cost, sc.rgbx, H, W, C, D, radius, sigma_s, sigma_r, bf16, nullptr, disp_int,
                                     disp_subpix, ctx->derr, ctx->num_sms, st, 0, ctx->wait_cycles);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tensor-core aggregation launch");
    return FBS_OK;
}

}  // namespace fbs

namespace {

// The device address of a page-locked host buffer, or nullptr when the GPU
// cannot address it (pageable memory).
const void* device_view(const void* p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

fbs_status run_path(fbs_ctx* ctx, const uint8_t* left, const uint8_t* right, int H, int W, int C, int D,
                    int radius, float sigma_s, float sigma_r, float tau, int32_t* disp_int,
                    float* disp_subpix, cudaStream_t st)
{
    if (ctx->opt.prec != FBS_PREC_F32)
        return fbs::run_path_tc(ctx, left, right, H, W, C, D, radius, sigma_s, sigma_r, tau, disp_int, disp_subpix,
                                st);
    fbs_status inj = take_injected_failure(ctx);
    if (inj != FBS_OK) return inj;
    const int ld = fbs::padded_ld(D);
    const size_t stats = fbs::cost_scratch_bytes(H, W);
    const size_t need = stats + sizeof(float) * (size_t)H * W * ld;
    fbs_status s = ensure(ctx, &ctx->ws, &ctx->ws_bytes, need, "cost volume");
    if (s != FBS_OK) return s;
    const fbs::CostScratch sc = fbs::carve_cost_scratch(ctx->ws, H, W);
    float* cost = (float*)((uint8_t*)ctx->ws + stats);
    cudaError_t e;
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

}  // namespace

namespace fbs {

fbs_status check_path_args(fbs_ctx* ctx, const uint8_t* left, const uint8_t* right, int H, int W, int C, int D,
                           int radius, float sigma_s, float sigma_r, float tau, const int32_t* disp_int,
                           const float* disp_subpix)
{
    if (!left || !right) return fail(ctx, FBS_ERR_INVALID_ARG, "null image pointer");
    if (!disp_int && !disp_subpix) return fail(ctx, FBS_ERR_INVALID_ARG, "both outputs are NULL");
    fbs_status s = check_shape(ctx, H, W, C, D);
    if (s == FBS_OK) s = check_agg_params(ctx, radius, sigma_s, sigma_r);
    if (s == FBS_OK) s = check_tau(ctx, tau);
    return s;
}


thread_local long long tl_kernel_launches = 0;

cudaError_t raise_smem_limit(const void* kernel, size_t bytes)
{
    struct Entry {
        const void* kernel;
        int device;
        size_t bytes;
    };
    static std::mutex mu;
    static std::vector<Entry> table;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    for (Entry& x : table)
        if (x.kernel == kernel && x.device == dev) {
            if (x.bytes >= bytes) return cudaSuccess;
            e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
            if (e == cudaSuccess) x.bytes = bytes;
            return e;
        }
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) table.push_back({kernel, dev, bytes});
    return e;
}

}  // namespace fbs

extern "C" {

void fbs_default_options(fbs_options* opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof *opt);
    opt->cost = FBS_COST_NCC;
    opt->prec = FBS_PREC_F32;
}

fbs_status fbs_create(fbs_ctx** out, const fbs_options* opt, int device)
{
    if (!out) return FBS_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return FBS_ERR_CUDA;
    }
    if (device < 0 || device >= n) return FBS_ERR_INVALID_ARG;
    fbs_ctx* ctx = new (std::nothrow) fbs_ctx();
    if (!ctx) return FBS_ERR_OOM;
    if (opt) {
        if (check_options(ctx, opt) != FBS_OK) {
            delete ctx;
            return FBS_ERR_INVALID_ARG;
        }
        ctx->opt = *opt;
    } else {
        fbs_default_options(&ctx->opt);
    }
    ctx->device = device;
    DeviceGuard g(device);
    if (!g.ok) {
        delete ctx;
        return FBS_ERR_CUDA;
    }
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return FBS_ERR_CUDA;
    }
    if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->sm_khz, cudaDevAttrClockRate, device) != cudaSuccess ||
        cudaMalloc(&ctx->derr, sizeof(int)) != cudaSuccess || cudaMemset(ctx->derr, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->derr) cudaFree(ctx->derr);
        cudaStreamDestroy(ctx->stream);
        delete ctx;
        return FBS_ERR_CUDA;
    }
    *out = ctx;
    return FBS_OK;
}

fbs_status fbs_destroy(fbs_ctx* ctx)
{
    if (!ctx) return FBS_OK;
    DeviceGuard g(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (auto& r : ctx->recs) {
        cudaEventSynchronize(r.b);
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : ctx->spare) cudaEventDestroy(e);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->io) cudaFree(ctx->io);
    if (ctx->derr) cudaFree(ctx->derr);
    for (auto& kv : ctx->bgraphs) drop_batch_graph(kv.second);
    for (int k = 0; k < 3; ++k) {
        if (ctx->bbranch[k]) cudaStreamDestroy(ctx->bbranch[k]);
        if (ctx->bjoin[k]) cudaEventDestroy(ctx->bjoin[k]);
    }
    if (ctx->bfork) cudaEventDestroy(ctx->bfork);
    if (ctx->aux) cudaFree(ctx->aux);
    if (ctx->bpairs) cudaFree(ctx->bpairs);
    if (ctx->bcounters) cudaFree(ctx->bcounters);
    for (int k = 0; k < 2; ++k) {
        if (ctx->bstage[k]) cudaFreeHost(ctx->bstage[k]);
        if (ctx->bstage_done[k]) cudaEventDestroy(ctx->bstage_done[k]);
    }
    fbs::band_free(ctx);
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return FBS_OK;
}

fbs_status fbs_set_options(fbs_ctx* ctx, const fbs_options* opt)
{
    if (!ctx || !opt) return fail(ctx, FBS_ERR_INVALID_ARG, "null context or options");
    fbs_status s = check_options(ctx, opt);
    if (s != FBS_OK) return s;
    ctx->opt = *opt;
    return FBS_OK;
}

fbs_status fbs_sync(fbs_ctx* ctx)
{
    if (!ctx) return FBS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronise");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pending error");
    int word = 0;
    e = cudaMemcpy(&word, ctx->derr, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "read kernel error word");
    if (word != 0) {
        cudaMemset(ctx->derr, 0, sizeof(int));
        return fail(ctx, FBS_ERR_TIMEOUT, "a bounded wait inside a kernel gave up (code %d); its outputs are invalid", word);
    }
    return FBS_OK;
}

fbs_status fbs_debug_fail_launches(fbs_ctx* ctx, int cuda_error, int count)
{
    if (!ctx) return FBS_ERR_INVALID_ARG;
    if (count < 0 || (count > 0 && cuda_error == (int)cudaSuccess))
        return fail(ctx, FBS_ERR_INVALID_ARG, "count %d must be >= 0 and the error non-zero", count);
    ctx->inject_error = cuda_error;
    ctx->inject_count = count;
    return FBS_OK;
}

fbs_status fbs_set_wait_limit(fbs_ctx* ctx, double seconds)
{
    if (!ctx) return FBS_ERR_INVALID_ARG;
    if (!(seconds >= 0.0 && seconds <= 60.0))
        return fail(ctx, FBS_ERR_INVALID_ARG, "wait limit %g s outside 0 .. 60", seconds);
    ctx->wait_cycles = seconds == 0.0 ? 0 : std::max(1LL, (long long)(seconds * ctx->sm_khz * 1e3));
    return FBS_OK;
}

const char* fbs_last_error(const fbs_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

fbs_status fbs_profile(fbs_ctx* ctx, int enable)
{
    if (!ctx) return FBS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (enable) {
        for (auto& r : ctx->recs) {
            cudaEventSynchronize(r.b);
            ctx->spare.push_back(r.a);
            ctx->spare.push_back(r.b);
        }
        ctx->recs.clear();
        for (auto& n : ctx->launches) n = 0;
    }
    ctx->profiling = enable != 0;
    return FBS_OK;
}

fbs_status fbs_profile_read(fbs_ctx* ctx, int kind, double* total_ms, long long* launches)
{
    if (!ctx || kind < 0 || kind >= FBS_KERNEL_KINDS) return fail(ctx, FBS_ERR_INVALID_ARG, "bad kernel kind");
    DeviceGuard g(ctx->device);
    double t = 0.0;
    for (auto& r : ctx->recs) {
        if (r.kind != kind) continue;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "profile event");
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "profile elapsed time");
        t += ms;
    }
    if (total_ms) *total_ms = t;
    if (launches) *launches = ctx->launches[kind];
    return FBS_OK;
}

fbs_status fbs_compute_disparity(fbs_ctx* ctx, const uint8_t* left, const uint8_t* right, int H, int W,
                                 int C, int D, int radius, float sigma_s, float sigma_r, float tau,
                                 int32_t* disp_int, float* disp_subpix, void* cuda_stream)
{
    if (!ctx) return FBS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!left || !right) return fail(ctx, FBS_ERR_INVALID_ARG, "null image pointer");
    if (!disp_int && !disp_subpix) return fail(ctx, FBS_ERR_INVALID_ARG, "both outputs are NULL");
    fbs_status s = check_shape(ctx, H, W, C, D);
    if (s == FBS_OK) s = check_agg_params(ctx, radius, sigma_s, sigma_r);
    if (s == FBS_OK) s = check_tau(ctx, tau);
    if (s != FBS_OK) return s;
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(ctx, FBS_ERR_CUDA, "cannot select device %d", ctx->device);
    return run_path(ctx, left, right, H, W, C, D, radius, sigma_s, sigma_r, tau, disp_int, disp_subpix,
                    pick_stream(ctx, cuda_stream));
}

fbs_status fbs_compute_disparity_host(fbs_ctx* ctx, const uint8_t* left, const uint8_t* right, int H, int W,
                                      int C, int D, int radius, float sigma_s, float sigma_r, float tau,
                                      int32_t* disp_int, float* disp_subpix)
{
    if (!ctx) return FBS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!left || !right) return fail(ctx, FBS_ERR_INVALID_ARG, "null image pointer");
    if (!disp_int && !disp_subpix) return fail(ctx, FBS_ERR_INVALID_ARG, "both outputs are NULL");
    fbs_status s = check_shape(ctx, H, W, C, D);
    if (s == FBS_OK) s = check_agg_params(ctx, radius, sigma_s, sigma_r);
    if (s == FBS_OK) s = check_tau(ctx, tau);
    if (s != FBS_OK) return s;
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(ctx, FBS_ERR_CUDA, "cannot select device %d", ctx->device);
    // Tensor-core form with page-locked host buffers the GPU can address: no
    // staging copies -- the cost kernel reads the images from host memory and
    // the aggregation epilogue writes the maps there (over the host link; only
    // these two kernels touch the caller's buffers, each byte once).
    if (ctx->opt.prec != FBS_PREC_F32) {
        const uint8_t *hl = (const uint8_t*)device_view(left), *hr = (const uint8_t*)device_view(right);
        int32_t* hi = disp_int ? (int32_t*)device_view(disp_int) : nullptr;
        float* hs = disp_subpix ? (float*)device_view(disp_subpix) : nullptr;
        if (hl && hr && (hi || !disp_int) && (hs || !disp_subpix)) {
            s = fbs::run_path_tc(ctx, hl, hr, H, W, C, D, radius, sigma_s, sigma_r, tau, hi, hs, ctx->stream);
            if (s != FBS_OK) return s;
            cudaError_t e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "host-buffer call");
            return FBS_OK;
        }
    }
    const size_t npx = (size_t)H * W;
    const size_t img = npx * C;
    const size_t img_al = (img + 255) & ~(size_t)255;
    const size_t out_al = (npx * 4 + 255) & ~(size_t)255;
    s = ensure(ctx, &ctx->io, &ctx->io_bytes, 2 * img_al + 2 * out_al, "host-path staging");
    if (s != FBS_OK) return s;
    uint8_t* dl = (uint8_t*)ctx->io;
    uint8_t* dr = dl + img_al;
    int32_t* di = (int32_t*)(dr + img_al);
    float* dsub = (float*)((uint8_t*)di + out_al);
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaMemcpyAsync(dl, left, img, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dr, right, img, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "host-to-device copy");
    s = run_path(ctx, dl, dr, H, W, C, D, radius, sigma_s, sigma_r, tau, disp_int ? di : nullptr,
                 disp_subpix ? dsub : nullptr, st);
    if (s != FBS_OK) return s;
    if (disp_int) e = cudaMemcpyAsync(disp_int, di, npx * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && disp_subpix) e = cudaMemcpyAsync(disp_subpix, dsub, npx * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "device-to-host copy");
    return FBS_OK;
}

fbs_status fbs_cost_volume(fbs_ctx* ctx, const uint8_t* left, const uint8_t* right, int H, int W, int C,
                           int D, float tau, float* cost_out, void* cuda_stream)
{
    if (!ctx) return FBS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!left || !right || !cost_out) return fail(ctx, FBS_ERR_INVALID_ARG, "null pointer");
    fbs_status s = check_shape(ctx, H, W, C, D);
    if (s == FBS_OK) s = check_tau(ctx, tau);
    if (s != FBS_OK) return s;
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(ctx, FBS_ERR_CUDA, "cannot select device %d", ctx->device);
    fbs_status s2 = ensure(ctx, &ctx->ws, &ctx->ws_bytes, fbs::cost_scratch_bytes(H, W), "cost statistics");
    if (s2 != FBS_OK) return s2;
    const fbs::CostScratch sc = fbs::carve_cost_scratch(ctx->ws, H, W);
    cudaStream_t st = pick_stream(ctx, cuda_stream);
    cudaError_t e;
    {
        LaunchScope ls(ctx, FBS_KERNEL_COST, st);
        e = fbs::launch_cost_build(sc, left, right, H, W, C, D, D, ctx->opt.cost, tau, cost_out, st);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cost build launch");
    return FBS_OK;
}

fbs_status fbs_aggregate(fbs_ctx* ctx, const float* cost, const uint8_t* guide, int H, int W, int C, int D,
                         int radius, float sigma_s, float sigma_r, float* agg_out, int32_t* disp_int,
                         float* disp_subpix, void* cuda_stream)
{
    if (!ctx) return FBS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!cost || !guide) return fail(ctx, FBS_ERR_INVALID_ARG, "null pointer");
    if (!agg_out && !disp_int && !disp_subpix) return fail(ctx, FBS_ERR_INVALID_ARG, "all outputs are NULL");
    fbs_status s = check_shape(ctx, H, W, C, D);
    if (s == FBS_OK) s = check_agg_params(ctx, radius, sigma_s, sigma_r);
    if (s != FBS_OK) return s;
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(ctx, FBS_ERR_CUDA, "cannot select device %d", ctx->device);
    cudaStream_t st = pick_stream(ctx, cuda_stream);
    cudaError_t e;
    if (ctx->opt.prec != FBS_PREC_F32) {
        if (!fbs::tc_supported(D, radius))
            return fail(ctx, FBS_ERR_UNSUPPORTED, "tensor-core aggregation supports D <= 256 and radius <= 24");
        const bool bf16 = ctx->opt.prec == FBS_PREC_BF16;
        const size_t rgbx = fbs::rgbx_bytes(H, W);
        fbs_status s2 = ensure(ctx, &ctx->ws, &ctx->ws_bytes, rgbx + fbs::xblock16_bytes(H, W, D), "16-bit cost copy");
        if (s2 != FBS_OK) return s2;
        uint2* packed = (uint2*)ctx->ws;
        void* cost16 = (uint8_t*)ctx->ws + rgbx;
        {
            LaunchScope ls(ctx, FBS_KERNEL_OTHER, st);
            e = fbs::launch_hwd_to_xblock16(cost, H, W, D, bf16, cost16, st);
            if (e == cudaSuccess) e = fbs::launch_xblock16_pad_rows(H, W, D, bf16, cost16, st);
            if (e == cudaSuccess) e = fbs::launch_pack_rgbx(guide, H, W, C, packed, st);
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cost conversion launch");
        {
            LaunchScope ls(ctx, FBS_KERNEL_AGG_TC, st);
            e = fbs::launch_aggregate_tc(cost16, packed, H, W, C, D, radius, sigma_s, sigma_r, bf16, agg_out,
                                         disp_int, disp_subpix, ctx->derr, ctx->num_sms, st, 0, ctx->wait_cycles);
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "tensor-core aggregation launch");
        return FBS_OK;
    }
    {
        LaunchScope ls(ctx, FBS_KERNEL_AGG_F32, st);
        e = fbs::launch_aggregate_f32(cost, D, guide, H, W, C, D, radius, sigma_s, sigma_r, agg_out, disp_int,
                                      disp_subpix, st);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "aggregation launch");
    return FBS_OK;
}

}  // extern "C"
