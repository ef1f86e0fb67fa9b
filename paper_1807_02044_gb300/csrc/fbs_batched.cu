// Batched form: many stereo pairs of uneven size, disparity range and radius
// in one call, replayed as one CUDA graph per batch shape.
//
// FP32 precision: one persistent launch per stage (statistics, cost volumes,
// FP32 aggregation with WTA and Eq. (10)).  Each stage's kernel walks a flat
// list of work items (rows, row segments or 32x4 tiles of every pair); CTAs
// claim items with an atomicAdd on a per-stage counter, so uneven pairs
// balance themselves and no CTA ever waits on another.  The graph is [copy
// the pair table from a pinned slot, reset the counters, three persistent
// launches]; device pointers are read from the table at run time, so one
// graph serves any buffers of that shape.  These plans differ in pair order
// (largest first or as given) and in aggregation CTAs per SM (1 or 2).
//
// Branched plans (every precision): each pair runs the launches of the
// single-pair form over its own slice of one scratch that holds every pair's
// volume -- FP32: statistics, cost volume, aggregation; BF16 / FP16: 16-bit
// cost volume (statistics, pad rows and packed guide in the same kernel),
// tcgen05 aggregation.  The graph has 1, 2
// or 4 independent branches; pairs go, largest first, to the branch with the
// least work so far, so one pair's memory-bound cost build overlaps another's
// aggregation and small pairs fill the SMs a large pair's last wave leaves
// idle.  Tensor-core plans also differ in the window rows per pipeline stage
// (the kernel's maximum, or at most 3: smaller stages, more of them).  The
// kernels' arguments (and the tensor maps) hold the pairs' addresses, so
// these graphs are keyed by the buffers too.
//
// Plan 6 of the tensor-core form keeps the per-pair cost builds (2 branches)
// and replaces the per-pair aggregations by persistent launches that walk
// the tiles of every pair, one launch per radius variant present in the batch
// (fbs_aggregate_tc_batch.cu).
//
// Either way each pair's results are bit-identical to fbs_compute_disparity
// in the same precision (the same kernels run on the same data in the same
// order).  The first call of a new shape (the list of H, W, C, D, radius, the
// cost mode and the precision) times each plan on the caller's data and keeps
// the fastest, appending "shape plan" to the autotune cache file when one is
// configured.
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
// FP32: plans 0-3 persistent, plan = 2 * order + (agg CTAs per SM - 1), order 0
// = largest first; plans 4-6 branched with kBranches[plan - 4] branches.
constexpr int kPersistentPlans = 4;
constexpr int kPlans = 7;
// tensor cores: plans 0-5 = 2 * branch choice + stage choice; plan 6 the
// cost builds on 2 branches, then persistent aggregations over every pair's
// tiles (one launch per radius variant)
constexpr int kTcPersistentPlan = 6;
constexpr int kTcPlans = 7;
constexpr int kBranches[3] = {1, 2, 4};
constexpr int kTcRowCap[2] = {0, 3};   // window rows per stage: 0 = the kernel's maximum
constexpr size_t kMaxBranchGraphs = 32;   // branched graphs kept for distinct buffer sets

bool tc_batch(const fbs_ctx* ctx) { return ctx->opt.prec != FBS_PREC_F32; }
int plan_count(const fbs_ctx* ctx) { return tc_batch(ctx) ? kTcPlans : kPlans; }

std::string batch_signature(fbs_ctx* ctx, int n, const fbs_pair* pairs)
{
    std::ostringstream os;
    // FP32 signatures keep their original form; tensor-core ones name the precision
    if (tc_batch(ctx)) os << (ctx->opt.prec == FBS_PREC_BF16 ? "tb" : "th");
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
        if (plan >= 0 && plan < (sig[0] == 't' ? kTcPlans : kPlans)) ctx->btuned[sig] = plan;
}

void store_tuned(fbs_ctx* ctx, const std::string& sig, int plan)
{
    if (!ctx->opt.autotune_cache_path) return;
    // a leading newline keeps the entry on a line of its own even after a
    // truncated last line (blank lines are skipped by load_tuned)
    std::ofstream f(ctx->opt.autotune_cache_path, std::ios::app);
    if (f) f << "\n" << sig << " " << plan << "\n";
}

// Device buffers that graphs capture by address: grown only here, and every
// graph is dropped when they move.
fbs_status ensure_batch_buffers(fbs_ctx* ctx, int n)
{
    if (ctx->bpairs && ctx->bpairs_cap >= n) return FBS_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronise before growing the batch table");
    for (auto& kv : ctx->bgraphs) drop_batch_graph(kv.second);
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

// work of one pair: pixels * disparities * window taps
double pair_work(const fbs_pair& q)
{
    const double t = (2.0 * q.radius + 1) * (2.0 * q.radius + 1);
    return (double)q.H * q.W * q.D * t;
}

std::vector<int> largest_first(int n, const fbs_pair* pairs)
{
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return pair_work(pairs[a]) > pair_work(pairs[b]); });
    return order;
}

Layout plan_layout(int n, const fbs_pair* pairs, int order_kind)
{
    Layout L;
    L.order.resize(n);
    std::iota(L.order.begin(), L.order.end(), 0);
    if (order_kind == 0) L.order = largest_first(n, pairs);
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
    ctx->launches[FBS_KERNEL_COST] += 2;   // statistics and cost
    ctx->launches[FBS_KERNEL_AGG_F32] += 1;
    return FBS_OK;
}

// ---- branched plans: every pair's single-pair launches in one graph ----------------

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Scratch of one pair.  Tensor cores: [packed guide | 16-bit x-blocked
// volume]; FP32: [statistics | FP32 volume, row pitch padded_ld(D)].
size_t pair_bytes(const fbs_pair& q, bool tc)
{
    if (!tc) return align256(fbs::cost_scratch_bytes(q.H, q.W)) +
                    align256(sizeof(float) * (size_t)q.H * q.W * fbs::padded_ld(q.D));
    return align256(fbs::rgbx_bytes(q.H, q.W)) + align256(fbs::xblock16_bytes(q.H, q.W, q.D));
}

fbs_status ensure_branches(fbs_ctx* ctx)
{
    cudaError_t e = cudaSuccess;
    if (!ctx->bfork) e = cudaEventCreateWithFlags(&ctx->bfork, cudaEventDisableTiming);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        if (!ctx->bbranch[k]) e = cudaStreamCreateWithFlags(&ctx->bbranch[k], cudaStreamNonBlocking);
        if (e == cudaSuccess && !ctx->bjoin[k]) e = cudaEventCreateWithFlags(&ctx->bjoin[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch branch streams");
    return FBS_OK;
}

// Capture every pair's launches of the single-pair form of the context's
// precision, spread over nb branches, into one graph (rows: the tensor-core
// stage cap).  With `persistent` (tensor cores) the graph holds only the
// pairs' cost builds on the branches and, after they join, the persistent
// aggregation launches over every pair's tiles (one per radius variant),
// whose pair table the graph owns.
fbs_status build_branch_graph(fbs_ctx* ctx, int n, const fbs_pair* pairs, int nb, int rows, bool persistent,
                              fbs_batch_graph* g)
{
    const bool tc = tc_batch(ctx);
    const bool bf16 = ctx->opt.prec == FBS_PREC_BF16;
    const int mode = ctx->opt.cost;
    fbs_status st = ensure_branches(ctx);
    if (st != FBS_OK) return st;
    const std::vector<int> order = largest_first(n, pairs);
    fbs::TcBatchLaunch tcl{};
    if (persistent) {
        // the pair table (tensor maps of each pair's slice of the scratch) is
        // built and uploaded before the capture
        std::vector<fbs::TcBatchMember> mem(n);
        size_t off = 0;
        for (int k = 0; k < n; ++k) {
            const fbs_pair& q = pairs[order[k]];
            uint8_t* base = (uint8_t*)ctx->ws + off;
            off += pair_bytes(q, true);
            mem[k] = fbs::TcBatchMember{base + align256(fbs::rgbx_bytes(q.H, q.W)), (const uint2*)base, q.H, q.W, q.C,
                                        q.D, q.radius, q.sigma_s, q.sigma_r, q.disp_int, q.disp_subpix};
        }
        std::vector<uint8_t> host(fbs::tc_batch_table_bytes(n));
        cudaError_t e = fbs::tc_batch_prepare(n, mem.data(), bf16, host.data(), &tcl);
        if (e == cudaSuccess) e = cudaMalloc(&g->table, host.size());
        if (e == cudaSuccess) e = cudaMemcpy(g->table, host.data(), host.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            if (g->table) cudaFree(g->table);
            g->table = nullptr;
            return cuda_fail(ctx, e, "persistent batch pair table");
        }
    }
    cudaStream_t cs = ctx->stream;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "begin graph capture");
    if (nb > 1) e = cudaEventRecord(ctx->bfork, cs);
    int joined = 0;   // branches that joined the capture (each must be joined back)
    for (int k = 1; k < nb && e == cudaSuccess; ++k) {
        e = cudaStreamWaitEvent(ctx->bbranch[k - 1], ctx->bfork, 0);
        if (e == cudaSuccess) joined = k;
    }
    std::vector<double> load(nb, 0.0);
    size_t off = 0;
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        const fbs_pair& q = pairs[order[k]];
        const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[b] += pair_work(q);
        cudaStream_t s = b == 0 ? cs : ctx->bbranch[b - 1];
        uint8_t* base = (uint8_t*)ctx->ws + off;
        off += pair_bytes(q, tc);
        long long k0 = fbs::launch_count();
        if (!tc) {
            const size_t stats = align256(fbs::cost_scratch_bytes(q.H, q.W));
            const fbs::CostScratch sc = fbs::carve_cost_scratch(base, q.H, q.W);
            const int ld = fbs::padded_ld(q.D);
            float* cost = (float*)(base + stats);
            e = fbs::launch_cost_build(sc, q.left, q.right, q.H, q.W, q.C, q.D, ld, mode, q.tau, cost, s);
            g->kernels[FBS_KERNEL_COST] += fbs::launch_count() - k0;
            k0 = fbs::launch_count();
            if (e == cudaSuccess)
                e = fbs::launch_aggregate_f32(cost, ld, q.left, q.H, q.W, q.C, q.D, q.radius, q.sigma_s, q.sigma_r,
                                              nullptr, q.disp_int, q.disp_subpix, s);
            g->kernels[FBS_KERNEL_AGG_F32] += fbs::launch_count() - k0;
            continue;
        }
        fbs::CostScratch sc{};
        sc.rgbx = (uint2*)base;
        void* cost = base + align256(fbs::rgbx_bytes(q.H, q.W));
        e = fbs::launch_cost_build_xblock16(sc, q.left, q.right, q.H, q.W, q.C, q.D, mode, q.tau, bf16, cost, s);
        g->kernels[FBS_KERNEL_COST] += fbs::launch_count() - k0;
        k0 = fbs::launch_count();
        if (e == cudaSuccess && !persistent)
            e = fbs::launch_aggregate_tc(cost, sc.rgbx, q.H, q.W, q.C, q.D, q.radius, q.sigma_s, q.sigma_r, bf16,
                                         nullptr, q.disp_int, q.disp_subpix, ctx->derr, ctx->num_sms, s, rows,
                                         ctx->wait_cycles);
        g->kernels[FBS_KERNEL_AGG_TC] += fbs::launch_count() - k0;
    }
    // join every branch back, also after a failed launch, so the capture ends cleanly
    for (int k = 1; k <= joined; ++k) {
        cudaError_t e1 = cudaEventRecord(ctx->bjoin[k - 1], ctx->bbranch[k - 1]);
        if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(cs, ctx->bjoin[k - 1], 0);
        if (e == cudaSuccess) e = e1;
    }
    if (persistent && e == cudaSuccess) {
        const long long k0 = fbs::launch_count();
        e = fbs::launch_aggregate_tc_batch(g->table, tcl, bf16, ctx->derr, ctx->num_sms, ctx->wait_cycles, cs);
        g->kernels[FBS_KERNEL_AGG_TC] += fbs::launch_count() - k0;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->table) cudaFree(g->table);
        g->exec = nullptr;
        g->table = nullptr;
        return cuda_fail(ctx, e, "branched batch graph capture");
    }
    return FBS_OK;
}

fbs_status run_branch_plan(fbs_ctx* ctx, const std::string& sig, int n, const fbs_pair* pairs, int plan, int nb,
                           int rows, bool persistent, cudaStream_t stream)
{
    size_t need = 0;
    for (int i = 0; i < n; ++i) need += pair_bytes(pairs[i], tc_batch(ctx));
    fbs_status st = ensure(ctx, &ctx->ws, &ctx->ws_bytes, need, "batch cost volumes");
    if (st != FBS_OK) return st;
    // graphs that hold the pairs' addresses are keyed by them ("g|" prefix)
    std::ostringstream key;
    key << "g|" << sig << "|p" << plan << "|ws" << (uintptr_t)ctx->ws << std::hex;
    for (int i = 0; i < n; ++i)
        key << "|" << (uintptr_t)pairs[i].left << "," << (uintptr_t)pairs[i].right << ","
            << (uintptr_t)pairs[i].disp_int << "," << (uintptr_t)pairs[i].disp_subpix;
    auto it = ctx->bgraphs.find(key.str());
    if (it == ctx->bgraphs.end()) {
        size_t held = 0;
        for (auto& kv : ctx->bgraphs) held += kv.first.compare(0, 2, "g|") == 0;
        if (held >= kMaxBranchGraphs) {
            // too many buffer sets: drop the branched graphs (none is in use on the host side)
            cudaError_t e = cudaStreamSynchronize(stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronise before dropping batch graphs");
            for (auto g = ctx->bgraphs.begin(); g != ctx->bgraphs.end();) {
                if (g->first.compare(0, 2, "g|") == 0) {
                    drop_batch_graph(g->second);
                    g = ctx->bgraphs.erase(g);
                } else {
                    ++g;
                }
            }
        }
        fbs_batch_graph g;
        st = build_branch_graph(ctx, n, pairs, nb, rows, persistent, &g);
        if (st != FBS_OK) return st;
        it = ctx->bgraphs.emplace(key.str(), g).first;
    }
    cudaError_t e = cudaGraphLaunch(it->second.exec, stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "branched batch graph launch");
    for (int k = 0; k < FBS_KERNEL_KINDS; ++k) ctx->launches[k] += it->second.kernels[k];
    return FBS_OK;
}

fbs_status run_any_plan(fbs_ctx* ctx, const std::string& sig, int n, const fbs_pair* pairs, int plan,
                        cudaStream_t stream)
{
    if (tc_batch(ctx)) {
        if (plan == kTcPersistentPlan) return run_branch_plan(ctx, sig, n, pairs, plan, 2, 0, true, stream);
        return run_branch_plan(ctx, sig, n, pairs, plan, kBranches[plan >> 1], kTcRowCap[plan & 1], false, stream);
    }
    if (plan < kPersistentPlans) return run_plan(ctx, sig, n, pairs, plan, stream);
    return run_branch_plan(ctx, sig, n, pairs, plan, kBranches[plan - kPersistentPlans], 0, false, stream);
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
    if (tc_batch(ctx))
        for (int i = 0; i < n; ++i)
            if (!fbs::tc_supported(pairs[i].D, pairs[i].radius))
                return fail(ctx, FBS_ERR_UNSUPPORTED,
                            "pair %d: tensor-core aggregation supports D <= 256 and radius <= 24 (got D=%d, radius=%d)",
                            i, pairs[i].D, pairs[i].radius);
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
        for (int plan = 0; plan < plan_count(ctx) && st == FBS_OK; ++plan) {
            st = run_any_plan(ctx, sig, n, pairs, plan, stream);
            for (int rep = 0; rep < 3 && st == FBS_OK; ++rep) {
                cudaEventRecord(a, stream);
                st = run_any_plan(ctx, sig, n, pairs, plan, stream);
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
    if (tuned->second >= plan_count(ctx)) return fail(ctx, FBS_ERR_INVALID_ARG, "bad cached plan");
    // one timed scope around the graph; its kernels are counted per kind by the plan runners
    LaunchScope ls(ctx, FBS_KERNEL_BATCH, stream);
    return run_any_plan(ctx, sig, n, pairs, tuned->second, stream);
}

extern "C" fbs_status fbs_batch_plan(fbs_ctx* ctx, int n, const fbs_pair* pairs, int* plan)
{
    if (!ctx || !pairs || !plan || n < 1) return FBS_ERR_INVALID_ARG;
    if (!ctx->btuned_loaded) load_tuned(ctx);
    auto it = ctx->btuned.find(batch_signature(ctx, n, pairs));
    *plan = it == ctx->btuned.end() ? -1 : it->second;
    return FBS_OK;
}

extern "C" fbs_status fbs_batch_set_plan(fbs_ctx* ctx, int n, const fbs_pair* pairs, int plan)
{
    if (!ctx) return FBS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!pairs || n < 1 || n > kMaxPairs) return fail(ctx, FBS_ERR_INVALID_ARG, "batch of %d pairs (1..%d)", n, kMaxPairs);
    if (plan < 0 || plan >= plan_count(ctx))
        return fail(ctx, FBS_ERR_INVALID_ARG, "plan %d outside 0..%d for this precision", plan, plan_count(ctx) - 1);
    if (!ctx->btuned_loaded) load_tuned(ctx);
    ctx->btuned[batch_signature(ctx, n, pairs)] = plan;
    return FBS_OK;
}
