// Batched form: many stereo pairs of uneven size, disparity range and radius
// through one persistent launch per stage (statistics, cost volumes, FP32
// aggregation with WTA and Eq. (10)), replayed as one CUDA graph.
//
// Work decomposition: each stage's kernel walks a flat list of work items
// (rows, row segments or 32x4 tiles of every pair); CTAs claim items with an
// atomicAdd on a per-stage counter, so uneven pairs balance themselves and no
// CTA ever waits on another.  Each pair's results are bit-identical to
// fbs_compute_disparity in FP32 precision (the same tile code runs on the
// same data in the same order).
//
// Per batch shape (the list of H, W, C, D, radius and the cost mode) the
// library keeps a plan chosen by its own autotuner and one CUDA graph per
// pinned staging slot: [copy the pair table from the slot, reset the
// counters, three persistent launches].  Device pointers are read from the
// table at run time, so a graph serves any buffers of that shape.  The plan
// candidates differ in pair order (largest first or as given) and in the
// number of aggregation CTAs per SM (1 or 2); the first call of a new shape
// times each candidate on the caller's data and keeps the fastest, appending
// "shape plan" to the autotune cache file when one is configured.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <fstream>
#include <numeric>
#include <sstream>

#include "fbs_context.cuh"

using namespace fbs_detail;

namespace {

constexpr int kMaxPairs = 4096;
constexpr int kPlans = 4;   // plan = 2 * order + (agg CTAs per SM - 1); order 0 = largest first

std::string batch_signature(fbs_ctx* ctx, int n, const fbs_pair* pairs)
{
    std::ostringstream os;
    os << "m" << ctx->opt.cost << ";";
    for (int i = 0; i < n; ++i)
        os << pairs[i].H << "x" << pairs[i].W << "x" << pairs[i].C << "x" << pairs[i].D << "r" << pairs[i].radius
           << ";";
    return os.str();
}

void load_tuned(fbs_ctx* ctx)
{
    ctx->btuned_loaded = true;
    if (!ctx->opt.autotune_cache_path) return;
    std::ifstream f(ctx->opt.autotune_cache_path);
    std::string sig;
    int plan;
    while (f >> sig >> plan)
        if (plan >= 0 && plan < kPlans) ctx->btuned[sig] = plan;
}

void store_tuned(fbs_ctx* ctx, const std::string& sig, int plan)
{
    if (!ctx->opt.autotune_cache_path) return;
    std::ofstream f(ctx->opt.autotune_cache_path, std::ios::app);
    if (f) f << sig << " " << plan << "\n";
}

// Device buffers that graphs capture by address: grown only here, and every
// graph is dropped when they move.
fbs_status ensure_batch_buffers(fbs_ctx* ctx, int n)
{
    if (ctx->bpairs && ctx->bpairs_cap >= n) return FBS_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronise before growing the batch table");
    for (auto& kv : ctx->bgraphs) cudaGraphExecDestroy(kv.second.exec);
    ctx->bgraphs.clear();
    if (ctx->bpairs) cudaFree(ctx->bpairs);
    for (int k = 0; k < 2; ++k)
        if (ctx->bstage[k]) cudaFreeHost(ctx->bstage[k]);
    ctx->bpairs = nullptr;
    ctx->bstage[0] = ctx->bstage[1] = nullptr;
    const int cap = std::max(n, 64);
    e = cudaMalloc(&ctx->bpairs, sizeof(fbs::BatchPair) * cap);
    if (e == cudaSuccess && !ctx->bcounters) e = cudaMalloc(&ctx->bcounters, 4 * sizeof(int));
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaMallocHost(&ctx->bstage[k], sizeof(fbs::BatchPair) * cap);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k)
        if (!ctx->bstage_done[k]) e = cudaEventCreateWithFlags(&ctx->bstage_done[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, FBS_ERR_OOM, "batch table allocation: %s", cudaGetErrorString(e));
    }
    ctx->bpairs_cap = cap;
    return FBS_OK;
}

struct Layout {
    std::vector<int> order;   // table position -> caller's pair index
    size_t ws_bytes = 0;
    std::vector<size_t> off;  // per table position: offset of its statistics; cost follows
    int items[3] = {0, 0, 0};
    int max_radius = 0;
};

Layout plan_layout(int n, const fbs_pair* pairs, int order_kind)
{
    Layout L;
    L.order.resize(n);
    std::iota(L.order.begin(), L.order.end(), 0);
    if (order_kind == 0) {
        // largest first: work = pixels * disparities * window taps
        auto work = [&](int i) {
            const double t = (2.0 * pairs[i].radius + 1) * (2.0 * pairs[i].radius + 1);
            return (double)pairs[i].H * pairs[i].W * pairs[i].D * t;
        };
        std::stable_sort(L.order.begin(), L.order.end(), [&](int a, int b) { return work(a) > work(b); });
    }
    L.off.resize(n);
    for (int k = 0; k < n; ++k) {
        const fbs_pair& q = pairs[L.order[k]];
        L.off[k] = L.ws_bytes;
        const size_t cost = (sizeof(float) * (size_t)q.H * q.W * fbs::padded_ld(q.D) + 255) & ~(size_t)255;
        L.ws_bytes += fbs::cost_scratch_bytes(q.H, q.W) + cost;
        L.items[0] += fbs::stats_items(q.H, q.W);
        L.items[1] += fbs::cost_items(q.H, q.W);
        L.items[2] += fbs::agg_f32_tiles(q.H, q.W);
        L.max_radius = std::max(L.max_radius, q.radius);
    }
    return L;
}

void fill_table(fbs_ctx* ctx, const Layout& L, int n, const fbs_pair* pairs, fbs::BatchPair* t)
{
    const double log2e = 1.4426950408889634;
    int so = 0, co = 0, ao = 0;
    for (int k = 0; k < n; ++k) {
        const fbs_pair& q = pairs[L.order[k]];
        fbs::BatchPair& b = t[k];
        b.left = q.left;
        b.right = q.right;
        b.H = q.H;
        b.W = q.W;
        b.C = q.C;
        b.D = q.D;
        b.radius = q.radius;
        b.ld = fbs::padded_ld(q.D);
        b.mode = ctx->opt.cost;
        b.neg_ks = (float)(-log2e / ((double)q.sigma_s * q.sigma_s));
        b.neg_kr = (float)(-log2e / ((double)q.sigma_r * q.sigma_r));
        b.tau = q.tau;
        uint8_t* base = (uint8_t*)ctx->ws + L.off[k];
        b.sc = fbs::carve_cost_scratch(base, q.H, q.W);
        b.cost = (float*)(base + fbs::cost_scratch_bytes(q.H, q.W));
        b.disp_int = q.disp_int;
        b.disp_sub = q.disp_subpix;
        b.stat_off = so;
        b.cost_off = co;
        b.agg_off = ao;
        so += fbs::stats_items(q.H, q.W);
        co += fbs::cost_items(q.H, q.W);
        ao += fbs::agg_f32_tiles(q.H, q.W);
    }
}

// Capture [table copy, counter reset, three persistent launches] for one plan and slot.
fbs_status build_graph(fbs_ctx* ctx, const Layout& L, int n, int plan, int slot, cudaGraphExec_t* out)
{
    size_t agg_smem = 0;
    cudaError_t e = fbs::prepare_aggregate_f32_batched(L.max_radius, &agg_smem);
    if (e == cudaSuccess) e = fbs::prepare_cost_batched();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batched kernel attributes");
    const int agg_per_sm = (plan & 1) + 1;
    const int g_stats = std::min(L.items[0], ctx->num_sms * 4);
    const int g_cost = std::min(L.items[1], ctx->num_sms * 4);
    const int g_agg = std::min(L.items[2], ctx->num_sms * agg_per_sm);
    cudaStream_t cs = ctx->stream;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "begin graph capture");
    e = cudaMemcpyAsync(ctx->bpairs, ctx->bstage[slot], sizeof(fbs::BatchPair) * n, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->bcounters, 0, 4 * sizeof(int), cs);
    if (e == cudaSuccess) e = fbs::launch_stats_batched(ctx->bpairs, n, L.items[0], ctx->bcounters + 0, g_stats, cs);
    if (e == cudaSuccess) e = fbs::launch_cost_batched(ctx->bpairs, n, L.items[1], ctx->bcounters + 1, g_cost, cs);
    if (e == cudaSuccess)
        e = fbs::launch_aggregate_f32_batched(ctx->bpairs, n, L.items[2], ctx->bcounters + 2, g_agg, agg_smem, cs);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batched graph capture");
    return FBS_OK;
}

fbs_status get_graph(fbs_ctx* ctx, const std::string& sig, const Layout& L, int n, int plan, int slot,
                     cudaGraphExec_t* out)
{
    const std::string key = sig + "|p" + std::to_string(plan) + "|s" + std::to_string(slot);
    auto it = ctx->bgraphs.find(key);
    if (it != ctx->bgraphs.end()) {
        *out = it->second.exec;
        return FBS_OK;
    }
    fbs_status st = build_graph(ctx, L, n, plan, slot, out);
    if (st != FBS_OK) return st;
    ctx->bgraphs[key] = fbs_batch_graph{*out, slot};
    return FBS_OK;
}

// Stage the table in the next pinned slot and launch the plan's graph on `stream`.
fbs_status run_plan(fbs_ctx* ctx, const std::string& sig, int n, const fbs_pair* pairs, int plan, cudaStream_t stream)
{
    const Layout L = plan_layout(n, pairs, plan >> 1);
    fbs_status st = ensure(ctx, &ctx->ws, &ctx->ws_bytes, L.ws_bytes, "batch cost volumes");
    if (st != FBS_OK) return st;
    const int slot = ctx->bslot;
    ctx->bslot ^= 1;
    cudaError_t e = cudaEventSynchronize(ctx->bstage_done[slot]);   // the slot's previous copy is done
    if (e != cudaSuccess) return cuda_fail(ctx, e, "wait for a staging slot");
    cudaGraphExec_t exec = nullptr;
    st = get_graph(ctx, sig + "|ws" + std::to_string((uintptr_t)ctx->ws), L, n, plan, slot, &exec);
    if (st != FBS_OK) return st;
    fill_table(ctx, L, n, pairs, ctx->bstage[slot]);
    e = cudaGraphLaunch(exec, stream);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->bstage_done[slot], stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batched graph launch");
    return FBS_OK;
}

}  // namespace

extern "C" fbs_status fbs_compute_disparity_batched(fbs_ctx* ctx, int n, const fbs_pair* pairs, void* cuda_stream)
{
    if (!ctx) return FBS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (n < 1 || n > kMaxPairs || !pairs) return fail(ctx, FBS_ERR_INVALID_ARG, "batch of %d pairs (1..%d)", n, kMaxPairs);
    for (int i = 0; i < n; ++i) {
        const fbs_pair& q = pairs[i];
        fbs_status s = fbs::check_path_args(ctx, q.left, q.right, q.H, q.W, q.C, q.D, q.radius, q.sigma_s, q.sigma_r,
                                            q.tau, q.disp_int, q.disp_subpix);
        if (s != FBS_OK) {
            std::string m = "pair " + std::to_string(i) + ": " + ctx->err;
            return fail(ctx, s, "%s", m.c_str());
        }
    }
    if (ctx->opt.prec != FBS_PREC_F32)
        return fail(ctx, FBS_ERR_UNSUPPORTED, "the batched form runs the FP32 aggregation only");
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(ctx, FBS_ERR_CUDA, "cannot select device %d", ctx->device);
    fbs_status st = ensure_batch_buffers(ctx, n);
    if (st != FBS_OK) return st;
    if (!ctx->btuned_loaded) load_tuned(ctx);
    cudaStream_t stream = pick_stream(ctx, cuda_stream);
    const std::string sig = batch_signature(ctx, n, pairs);

    auto tuned = ctx->btuned.find(sig);
    if (tuned == ctx->btuned.end()) {
        // autotune: time every plan on this batch (one warm-up, then the best of three)
        cudaEvent_t a = nullptr, b = nullptr;
        cudaError_t e = cudaEventCreate(&a);
        if (e == cudaSuccess) e = cudaEventCreate(&b);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune events");
        int best = 0;
        float best_ms = 1e30f;
        for (int plan = 0; plan < kPlans && st == FBS_OK; ++plan) {
            st = run_plan(ctx, sig, n, pairs, plan, stream);
            for (int rep = 0; rep < 3 && st == FBS_OK; ++rep) {
                cudaEventRecord(a, stream);
                st = run_plan(ctx, sig, n, pairs, plan, stream);
                cudaEventRecord(b, stream);
                e = cudaEventSynchronize(b);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
                if (e != cudaSuccess) st = cuda_fail(ctx, e, "autotune timing");
                if (st == FBS_OK && ms < best_ms) {
                    best_ms = ms;
                    best = plan;
                }
            }
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        if (st != FBS_OK) return st;
        ctx->btuned[sig] = best;
        store_tuned(ctx, sig, best);
        tuned = ctx->btuned.find(sig);
    }
    {
        LaunchScope ls(ctx, FBS_KERNEL_BATCH, stream);
        st = run_plan(ctx, sig, n, pairs, tuned->second, stream);
    }
    ctx->launches[FBS_KERNEL_COST] += 2;   // the batch graph runs three kernels
    ctx->launches[FBS_KERNEL_AGG_F32] += 1;
    ctx->launches[FBS_KERNEL_BATCH] -= 1;
    return st;
}

extern "C" fbs_status fbs_batch_plan(fbs_ctx* ctx, int n, const fbs_pair* pairs, int* plan)
{
    if (!ctx || !pairs || !plan || n < 1) return FBS_ERR_INVALID_ARG;
    if (!ctx->btuned_loaded) load_tuned(ctx);
    auto it = ctx->btuned.find(batch_signature(ctx, n, pairs));
    *plan = it == ctx->btuned.end() ? -1 : it->second;
    return FBS_OK;
}
