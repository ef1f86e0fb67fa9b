// Private definition of the library context and the host helpers shared by
// the translation units that implement the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "fbs.h"
#include "fbs_internal.cuh"

// One cached batch: the work description uploaded from a pinned staging slot
// and the CUDA graph that runs it.
struct fbs_batch_graph {
    cudaGraphExec_t exec = nullptr;
    int slot = 0;
    long long kernels[FBS_KERNEL_KINDS] = {};   // kernels one replay runs, per kind
    void* table = nullptr;                      // device pair table the graph's kernels read (if any)
};

// Release a batch graph and what it owns (the caller has synchronised).
inline void drop_batch_graph(fbs_batch_graph& g)
{
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.table) cudaFree(g.table);
    g.exec = nullptr;
    g.table = nullptr;
}

struct fbs_ctx {
    int device = 0;
    fbs_options opt{};
    cudaStream_t stream = nullptr;
    void* ws = nullptr;          // cost volume scratch
    size_t ws_bytes = 0;
    void* io = nullptr;          // device staging for the host-buffer entry point
    size_t io_bytes = 0;
    std::string err;
    int num_sms = 0;
    int* derr = nullptr;         // device error word written by kernels with bounded waits
    int sm_khz = 0;              // peak SM clock (kHz): converts the wait limit to clock cycles
    long long wait_cycles = 0;   // limit of one pipeline wait in the kernels (0 = their default, ~2 s)
    int inject_error = 0;        // failure injection: the cudaError_t the next steps report ...
    int inject_count = 0;        // ... for this many steps, instead of launching
    // kernel accounting
    long long launches[FBS_KERNEL_KINDS] = {};
    bool profiling = false;
    struct Rec {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;            // recorded launches since fbs_profile(ctx, 1)
    std::vector<cudaEvent_t> spare;   // event pool
    // batched form
    fbs::BatchPair* bpairs = nullptr;      // device pair table
    int bpairs_cap = 0;
    int* bcounters = nullptr;              // work counters of the three batched kernels
    fbs::BatchPair* bstage[2] = {nullptr, nullptr};   // pinned staging slots for the table
    cudaEvent_t bstage_done[2] = {nullptr, nullptr};  // slot free again when recorded work completes
    int bslot = 0;
    std::map<std::string, int> btuned;                 // batch shape -> chosen plan
    std::map<std::string, fbs_batch_graph> bgraphs;    // plan-specific graph per slot
    bool btuned_loaded = false;
    cudaStream_t bbranch[3] = {nullptr, nullptr, nullptr};   // extra branches of the tensor-core batch graph
    cudaEvent_t bfork = nullptr;
    cudaEvent_t bjoin[3] = {nullptr, nullptr, nullptr};
    // band form: the network's state and the band scratch (grown on demand)
    struct fbs_band_state* band = nullptr;
    void* band_ws = nullptr;
    size_t band_ws_bytes = 0;
    // both-view tensor-core form: mirrored images and right-view maps
    void* aux = nullptr;
    size_t aux_bytes = 0;
};

namespace fbs_detail {


struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

inline fbs_status fail(fbs_ctx* ctx, fbs_status st, const char* fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

inline fbs_status cuda_fail(fbs_ctx* ctx, cudaError_t e, const char* where)
{
    if (e == cudaErrorMemoryAllocation) return fail(ctx, FBS_ERR_OOM, "%s: %s", where, cudaGetErrorString(e));
    return fail(ctx, FBS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

// A step armed by fbs_debug_fail_launches reports the injected error instead
// of launching anything.
inline fbs_status take_injected_failure(fbs_ctx* ctx)
{
    if (ctx->inject_count <= 0) return FBS_OK;
    --ctx->inject_count;
    return cuda_fail(ctx, (cudaError_t)ctx->inject_error, "kernel launch (injected failure)");
}

inline bool finite_pos(float v) { return std::isfinite(v) && v > 0.f; }

inline fbs_status check_shape(fbs_ctx* ctx, int H, int W, int C, int D)
{
    if (H < 1 || H > 16384 || W < 1 || W > 16384)
        return fail(ctx, FBS_ERR_INVALID_ARG, "image size %dx%d outside 1..16384", W, H);
    if (C != 1 && C != 3) return fail(ctx, FBS_ERR_INVALID_ARG, "channels C=%d must be 1 or 3", C);
    if (D < 1 || D > 1024) return fail(ctx, FBS_ERR_INVALID_ARG, "disparity count D=%d outside 1..1024", D);
    return FBS_OK;
}

inline fbs_status check_agg_params(fbs_ctx* ctx, int radius, float sigma_s, float sigma_r)
{
    if (radius < 0 || radius > 31) return fail(ctx, FBS_ERR_INVALID_ARG, "radius=%d outside 0..31", radius);
    if (!finite_pos(sigma_s)) return fail(ctx, FBS_ERR_INVALID_ARG, "sigma_s must be finite and > 0");
    if (!finite_pos(sigma_r)) return fail(ctx, FBS_ERR_INVALID_ARG, "sigma_r must be finite and > 0");
    return FBS_OK;
}

inline fbs_status check_tau(fbs_ctx* ctx, float tau)
{
    if (ctx->opt.cost == FBS_COST_TAD && !(std::isfinite(tau) && tau >= 0.f))
        return fail(ctx, FBS_ERR_INVALID_ARG, "tau must be finite and >= 0 in TAD mode");
    return FBS_OK;
}

inline fbs_status check_options(fbs_ctx* ctx, const fbs_options* o)
{
    if (o->cost != FBS_COST_NCC && o->cost != FBS_COST_TAD)
        return fail(ctx, FBS_ERR_INVALID_ARG, "unknown cost mode %d", o->cost);
    if (o->prec != FBS_PREC_F32 && o->prec != FBS_PREC_BF16 && o->prec != FBS_PREC_F16)
        return fail(ctx, FBS_ERR_INVALID_ARG, "unknown precision %d", o->prec);
    return FBS_OK;
}

inline cudaStream_t pick_stream(fbs_ctx* ctx, void* s) { return s ? (cudaStream_t)s : ctx->stream; }

inline cudaEvent_t take_event(fbs_ctx* ctx)
{
    if (!ctx->spare.empty()) {
        cudaEvent_t e = ctx->spare.back();
        ctx->spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Bracket the kernel launches of one step for the accounting API (events
// around them when profiling; the number of kernels they launched).
// NVTX range names of the kernel kinds (host-side trace of each stage; the
// calls cost a few nanoseconds when no tracing tool is attached).
inline const char* kind_range_name(int kind)
{
    static const char* const names[FBS_KERNEL_KINDS] = {"fbs cost build", "fbs aggregation fp32",
                                                        "fbs aggregation tensor core", "fbs other",
                                                        "fbs batch graph", "fbs band network"};
    return kind >= 0 && kind < FBS_KERNEL_KINDS ? names[kind] : "fbs";
}

struct LaunchScope {
    fbs_ctx* ctx;
    int kind;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    long long k0 = fbs::launch_count();   // kernels noted inside the scope are counted
    LaunchScope(fbs_ctx* c, int k, cudaStream_t s) : ctx(c), kind(k), st(s)
    {
        nvtxRangePushA(kind_range_name(kind));
        if (ctx->profiling) {
            a = take_event(ctx);
            if (a) cudaEventRecord(a, st);
        }
    }
    ~LaunchScope()
    {
        nvtxRangePop();
        ctx->launches[kind] += fbs::launch_count() - k0;
        if (a) {
            cudaEvent_t b = take_event(ctx);
            if (b) {
                cudaEventRecord(b, st);
                ctx->recs.push_back({kind, a, b});
            } else {
                ctx->spare.push_back(a);
            }
        }
    }
};

// Grow-only device scratch, bounded by the context's cap.
inline fbs_status ensure(fbs_ctx* ctx, void** buf, size_t* have, size_t need, const char* what)
{
    if (need <= *have) return FBS_OK;
    const size_t cap = ctx->opt.workspace_cap;
    if (cap && ctx->ws_bytes + ctx->io_bytes + ctx->band_ws_bytes + ctx->aux_bytes - *have + need > cap)
        return fail(ctx, FBS_ERR_OOM, "%s needs %zu bytes; workspace cap is %zu", what, need, cap);
    if (*buf) {
        cudaError_t e = cudaDeviceSynchronize();   // the old buffer may still be in use
        if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronise before growing scratch");
        cudaFree(*buf);
        *buf = nullptr;
        *have = 0;
    }
    cudaError_t e = cudaMalloc(buf, need);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        return fail(ctx, FBS_ERR_OOM, "cudaMalloc(%zu) for %s: %s", need, what, cudaGetErrorString(e));
    }
    *have = need;
    return FBS_OK;
}

}  // namespace fbs_detail
