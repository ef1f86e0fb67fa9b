// Steps 2-4 of fast bilateral stereo on the tensor cores for a batch of
// uneven pairs: one persistent launch per group of members that share the
// producers' column-pair variant (a function of the radius).
//
// The work of a group is a flat list of tiles (16 x 8 pixels) over all its
// members, ordered by the work of one tile (largest first).  CTA b takes
// items b, b + grid, b + 2 grid, ...; every warp role walks that same
// sequence, so the roles agree on each tile without talking to one another
// and no CTA ever waits for another.  A tile is computed exactly as in the
// one-pair kernel -- the same weights (tc_weights), the same MMA sequence
// over the window rows and the same epilogue (tc_wta, tc_subpixel) -- so
// each pixel gets the bits of launch_aggregate_tc.
//
// What differs per member lives in a device table: the two tensor maps (cost
// volume, packed guide), the sizes, D, the radius, the constants of
// Eq. (7)-(8), the MMA instruction descriptors and the outputs.  The
// producers' column-pair code is specialised for the radius as in the
// one-pair kernel (kept inline: the same code behind a run-time switch over
// every variant, or behind calls, measured 1.3-1.6x slower), hence one kernel
// instance, and one launch, per variant present in the batch.
//
// Shared memory is laid out once per launch: S stages of a_stage bytes of
// weights and b_stage bytes of costs, sized for the group's largest member; a
// member with smaller rows puts more rows (its R) in a stage.  Weight
// positions a pixel never reaches must be zero.  Within a member they are
// never written, but a stage slot last filled by another member holds that
// member's weights, so a producer warp clears its own part of a slot before
// its first use by a new member.
#include <cuda.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "fbs_internal.cuh"
#include "tc_aggregate.cuh"

namespace fbs {
namespace {

using namespace tca;

// One member of the batch in the device table.
struct TcBatchPair {   // 128-byte aligned, as its tensor maps
    CUtensorMap tmap;       // 16-bit x-blocked cost volume; box 128 x Nb/16 x KW/8 x R
    CUtensorMap gmap;       // packed guide; box KW x NH
    int H, W, D, N, Nb, split, rho, rho8, KW, NH, ntx, R, variant;   // split: Nb > 256, two MMAs per K-step
    int item0, items;       // the member's tiles: work items item0 .. item0 + items - 1
    float neg_ks, neg_kr;
    uint32_t idesc, idesc2;   // the (first) MMA's instruction descriptor; the second one's when split
    int32_t* disp_int;
    float* disp_sub;
};

struct TcBatchArgs {
    const TcBatchPair* pairs;
    int npairs, nitems, S, nacc, kw_max, nh_max;
    uint32_t a_stage, b_stage, acc_stride, tmem_cols;
    long long wait_cycles;
};

struct BatchSmem {
    size_t a_off, b_off, g_off, bar_off, misc_off, own_off, total;
};

__host__ __device__ inline BatchSmem batch_smem_layout(int S, uint32_t a_stage, uint32_t b_stage, int kw_max,
                                                       int nh_max)
{
    BatchSmem s;
    size_t o = 0;
    s.a_off = o;
    o += (size_t)S * a_stage;
    s.b_off = o;
    o += (size_t)S * b_stage;
    o = (o + 127) & ~(size_t)127;
    s.g_off = o;
    o += (size_t)2 * nh_max * kw_max * 8;
    o = (o + 15) & ~(size_t)15;
    s.bar_off = o;
    o += (size_t)(3 * S + 9) * 8;
    s.misc_off = o;
    o += 16;
    s.own_off = o;        // per producer warp and stage slot: the member whose layout the slot holds
    o += (size_t)kProducerWarps * 8 * 4;
    s.total = o + 1024;   // slack for aligning the base to 1024 bytes
    return s;
}

// The instantiated producer variants: column pairs per thread and window row
// NPT = ceil((radius + 1) / 2) exact up to 8 with PM 0 (odd radius, every
// pair) or 1 (even radius, all but the last pair of phase 1), then NPT 10 and
// 13 with per-pair flags (PM 2) -- the same choice as the one-pair launch.
__host__ __device__ inline int batch_variant(int radius)
{
    const int npt = (radius + 2) / 2;
    if (npt <= 8) return 2 * (npt - 1) + ((radius & 1) ? 0 : 1);
    return npt <= 10 ? 16 : 17;
}

// Tile coordinates of work item `item` of member P.
__device__ __forceinline__ void tile_of(const TcBatchPair& P, int item, int& tx0, int& ty0)
{
    const int lt = item - P.item0;
    const int ty = lt / P.ntx;
    tx0 = (lt - ty * P.ntx) * kTW;
    ty0 = ty * kTH;
}

// Advance the member index to the member that holds `item` (items grow).
__device__ __forceinline__ int member_of(const TcBatchPair* pairs, int npairs, int pi, int item)
{
    while (pi + 1 < npairs && pairs[pi + 1].item0 <= item) ++pi;
    return pi;
}

// A member's fields as the TMA, MMA and epilogue roles use them, read from
// the table once per member (not once per tile).
struct MemberView {
    const TcBatchPair* p;
    int index, item0, end, ntx, H, W, D, N, Nb, split, rho, rho8, KW, NH, R;
    uint32_t idesc, idesc2;
    int32_t* disp_int;
    float* disp_sub;
};
__device__ __forceinline__ void view_member(MemberView& v, const TcBatchPair* pairs, int pi)
{
    const TcBatchPair& P = pairs[pi];
    v.p = &P;
    v.index = pi;
    v.item0 = P.item0;
    v.end = P.item0 + P.items;
    v.ntx = P.ntx;
    v.H = P.H;
    v.W = P.W;
    v.D = P.D;
    v.N = P.N;
    v.Nb = P.Nb;
    v.split = P.split;
    v.rho = P.rho;
    v.rho8 = P.rho8;
    v.KW = P.KW;
    v.NH = P.NH;
    v.R = P.R;
    v.idesc = P.idesc;
    v.idesc2 = P.idesc2;
    v.disp_int = P.disp_int;
    v.disp_sub = P.disp_sub;
}
// Tile coordinates of work item `item` of the viewed member.
__device__ __forceinline__ void tile_of(const MemberView& v, int item, int& tx0, int& ty0)
{
    const int lt = item - v.item0;
    const int ty = lt / v.ntx;
    tx0 = (lt - ty * v.ntx) * kTW;
    ty0 = ty * kTH;
}

extern __shared__ uint8_t tcb_smem_raw[];

// The launch's shared memory, aligned to 1024 bytes by an offset from the
// __shared__ array itself, so that every pointer derived from it is known to
// be a shared-memory one (32-bit shared loads and stores, not generic ones).
__device__ __forceinline__ uint8_t* batch_smem()
{
    return tcb_smem_raw + ((1024u - (smem_u32(tcb_smem_raw) & 1023u)) & 1023u);
}

// A producer warp's progress, carried from run to run.
struct ProducerState {
    int item;            // next work item of this CTA
    uint32_t t;          // tiles done (guide slot and parity)
    uint32_t gs, gu;     // stage slot and use count of the next stage
    int stop;            // the CTA has aborted
};

// The weights of the tiles item, item + grid, ... of member pi (all of them
// below the member's last item), with the column-pair code of the launch's
// variant (NPT, PM).  The lane and row mapping is the one-pair kernel's: warp w
// covers pixel rows 2 (w >> 2) and + 1 of the tile and the window rows r with
// r % 4 == w % 4 of every stage; lane -> pixel column xm = lane & 15 and pair
// phase h = lane >> 4.  Returns the warp's progress (stop set when the CTA
// has aborted).
template <bool BF16, int NPT, int PM>
__device__ __forceinline__ ProducerState produce_run(const TcBatchPair* __restrict__ pairs, int pi, ProducerState st,
                                                  const TcBatchArgs* __restrict__ a, int* __restrict__ err)
{
    uint8_t* sm = batch_smem();
    const BatchSmem L = batch_smem_layout(a->S, a->a_stage, a->b_stage, a->kw_max, a->nh_max);
    uint8_t* a_base = sm + L.a_off;
    const uint8_t* g_base = sm + L.g_off;
    const int S = a->S;
    const uint32_t a_stage = a->a_stage;
    const uint32_t g_slot = (uint32_t)a->nh_max * a->kw_max * 8;
    const uint32_t bars = smem_u32(sm + L.bar_off);
    const uint32_t full_a0 = bars, empty0 = bars + 16 * S, g_full0 = bars + 24 * S + 40, g_empty0 = g_full0 + 16;
    volatile uint32_t* abort_flag = (volatile uint32_t*)(sm + L.misc_off) + 1;
    const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
    volatile int* owner = (volatile int*)(sm + L.own_off) + 8 * warp;
    const long long wait = a->wait_cycles;
    const TcBatchPair& P = pairs[pi];
    const int rho = P.rho, KW = P.KW, NH = P.NH, H = P.H, W = P.W, R = P.R;
    const float neg_ks = P.neg_ks;
    const int ty = 2 * (warp >> 2), rq = warp & 3;
    const int xm = lane & 15, h = lane >> 4;
    const int m0 = 16 * ty + xm;
    const int kcen = xm + P.rho8;
    const int c0 = (kcen - rho) & ~1;
    const int np = rho + 1;
    bool on[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j)
        on[j] = PM == 0 ? true : PM == 1 ? (j < NPT - 1 || h == 0) : 2 * j + h < np;
    const TcPairOffsets po = tc_pair_offsets(c0 + 2 * h, m0);
    const uint32_t gcol = (uint32_t)(c0 + 2 * h) * 8;
    const uint32_t g_row = (uint32_t)KW * 8;
    const uint32_t a_row = (uint32_t)(KW / 8) * kALbo;
    const float ninf = __int_as_float(0xff800000);
    const uint64_t magic2 = f2_pack(-8388608.f, -8388608.f);
    const uint64_t nkr2 = f2_pack(P.neg_kr, P.neg_kr);
    const unsigned two_rho = (unsigned)(2 * rho);
    // spatial y-term of row offset i - rho, (ks dy^2, ks dy^2): the one-pair
    // kernel's table entry, computed per row (a table in global memory, or
    // one per warp in shared memory, measured slower)
    auto syt = [&](int i) -> uint64_t {
        const int dy = i - rho;
        const float sy = (float)(dy * dy) * neg_ks;
        return f2_pack(sy, sy);
    };
    const int end = P.item0 + P.items;
    for (; st.item < end; st.item += (int)gridDim.x, ++st.t) {
        int tx0, ty0;
        tile_of(P, st.item, tx0, ty0);
        const int xlo = tx0 - P.rho8;
        const uint32_t tb = st.t & 1;
        if (!mbar_wait_or_abort(g_full0 + 8 * tb, (st.t >> 1) & 1, abort_flag, wait)) {
            raise_abort(abort_flag, err, 6);
            st.stop = 1;
            return st;
        }
        const uint8_t* gt = g_base + tb * g_slot;
        const uint2 pc0 = *(const uint2*)(gt + (ty + rho) * g_row + kcen * 8);
        const uint2 pc1 = *(const uint2*)(gt + (ty + 1 + rho) * g_row + kcen * 8);
        const uint32_t pcol0 = pc0.x, pp0 = pc0.y + kMagic, pcol1 = pc1.x, pp1 = pc1.y + kMagic;
        uint64_t sxp[NPT];
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            const int k = c0 + 2 * h + 4 * j;
            const int d0 = k - kcen, d1 = d0 + 1;
            const int x0 = xlo + k;
            const float s0 = (d0 >= -rho && d0 <= rho && (unsigned)x0 < (unsigned)W) ? (float)(d0 * d0) * neg_ks : ninf;
            const float s1 =
                (d1 >= -rho && d1 <= rho && (unsigned)(x0 + 1) < (unsigned)W) ? (float)(d1 * d1) * neg_ks : ninf;
            sxp[j] = f2_pack(s0, s1);
        }
        const uint8_t* gth = gt + gcol;
        auto row_pairs = [&](uint8_t* arow, const uint8_t* grow, uint64_t sy0, uint64_t sy1, int which)
                             __attribute__((always_inline)) {
            tc_row_pairs<BF16, NPT>(arow, grow, po, on, sxp, sy0, sy1, which, pcol0, pp0, pcol1, pp1, magic2, nkr2);
        };
        const int hr_lo = max(0, rho - ty0);
        const int hr_hi = min(NH, H - ty0 + rho);
        for (int h0 = hr_lo; h0 < hr_hi; h0 += R) {
            const int nr = min(R, hr_hi - h0);
            const uint32_t s = st.gs, use = st.gu;
            bool ok = true;
            if (lane == 0 && use > 0) ok = mbar_wait_or_abort(empty0 + 8 * s, (use - 1) & 1, abort_flag, wait);
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
                raise_abort(abort_flag, err, 1);
                st.stop = 1;
                return st;
            }
            uint8_t* ast = a_base + s * a_stage;
            if (owner[s] != pi) {
                // the slot holds another member's layout: clear this warp's
                // pixel rows of its window rows before the first use
                const uint4 z = make_uint4(0u, 0u, 0u, 0u);
                for (int r = rq; r < R; r += 4)
                    for (int kb = h; kb < KW / 8; kb += 2) {
                        uint8_t* q = ast + r * a_row + kb * kALbo + m0 * 16;
                        *(uint4*)q = z;
                        *(uint4*)(q + 256) = z;
                    }
                __syncwarp();
                if (lane == 0) owner[s] = pi;
            }
#pragma unroll
            for (int r = rq; r < kMaxR; r += 4) {
                if (r >= nr) break;
                const int hr = h0 + r;
                const int dy = hr - ty;   // row offset + rho of the upper pixel
                const bool in0 = (unsigned)dy <= two_rho, in1 = (unsigned)(dy - 1) <= two_rho;
                uint8_t* arow = ast + r * a_row;
                const uint8_t* grow = gth + hr * g_row;
                if (in0 && in1)
                    row_pairs(arow, grow, syt(dy), syt(dy - 1), 3);
                else if (in0)
                    row_pairs(arow, grow, syt(dy), 0ull, 1);
                else if (in1)
                    row_pairs(arow, grow, 0ull, syt(dy - 1), 2);
                else
                    row_pairs(arow, grow, 0ull, 0ull, 0);
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(full_a0 + 8 * s);
            if (++st.gs == (uint32_t)S) {
                st.gs = 0;
                ++st.gu;
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(g_empty0 + 8 * tb);   // this tile's guide is no longer read
    }
    return st;
}

// Warp roles and pipeline as in the one-pair kernel: warps 0-15 weight
// producers, 16-19 epilogue (TMEM lane quarters), 20 TMA (guide tiles and
// cost rows), 21 MMA issuer; full_a / full_b / empty per stage slot,
// acc_full / acc_empty per accumulator buffer, g_full / g_empty per guide slot.
template <bool BF16, int NPT, int PM>
__global__ void __launch_bounds__(kThreads, 1)
aggregate_tc_batch_kernel(const __grid_constant__ TcBatchArgs a, int* __restrict__ err)
{
    uint8_t* sm = batch_smem();
    const BatchSmem L = batch_smem_layout(a.S, a.a_stage, a.b_stage, a.kw_max, a.nh_max);
    uint8_t* a_base = sm + L.a_off;
    uint8_t* b_base = sm + L.b_off;
    uint8_t* g_base = sm + L.g_off;
    const uint32_t g_slot = (uint32_t)a.nh_max * a.kw_max * 8;
    const int S = a.S;
    const uint32_t bars = smem_u32(sm + L.bar_off);
    const uint32_t full_a0 = bars, full_b0 = bars + 8 * S, empty0 = bars + 16 * S, acc_full0 = bars + 24 * S,
                   acc_empty0 = acc_full0 + 16, drain_bar = acc_empty0 + 16, g_full0 = drain_bar + 8,
                   g_empty0 = g_full0 + 16;
    uint32_t* misc = (uint32_t*)(sm + L.misc_off);   // [0] TMEM base, [1] abort flag
    volatile uint32_t* abort_flag = misc + 1;
    int* owners = (int*)(sm + L.own_off);
    const TcBatchPair* __restrict__ pairs = a.pairs;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grid = (int)gridDim.x;

    // ---- set-up --------------------------------------------------------------
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full_a0 + 8 * s, kProducerWarps);
            mbar_init(full_b0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(acc_full0 + 8 * s, 1);
            mbar_init(acc_empty0 + 8 * s, kEpilogue / 32);
            mbar_init(g_full0 + 8 * s, 1);
            mbar_init(g_empty0 + 8 * s, kProducerWarps);
        }
        mbar_init(drain_bar, 1);
        misc[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_u32(&misc[0]), a.tmem_cols);
    if (tid < kProducerWarps * 8) owners[tid] = -1;   // no slot holds a member's layout yet
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = misc[0];
    asm volatile("griddepcontrol.wait;" ::: "memory");

    if (warp < kProducerWarps) {
        // ================= weight producers =================================
        ProducerState st{(int)blockIdx.x, 0u, 0u, 0u, 0};
        int pi = 0;
        while (st.item < a.nitems && !st.stop) {
            pi = member_of(pairs, a.npairs, pi, st.item);
            st = produce_run<BF16, NPT, PM>(pairs, pi, st, &a, err);
        }
    } else if (warp < kTmaWarp) {
        // ================= epilogue: TMEM -> normalise -> WTA -> Eq. (10) ======
        const int q4 = warp - kEpiWarp0;
        const int m = 32 * q4 + lane;
        uint32_t t = 0;
        MemberView P;
        view_member(P, pairs, 0);
        for (int item = (int)blockIdx.x; item < a.nitems; item += grid, ++t) {
            if (item >= P.end) view_member(P, pairs, member_of(pairs, a.npairs, P.index, item));
            const uint32_t ab = a.nacc == 2 ? (t & 1) : 0, u = a.nacc == 2 ? (t >> 1) : t;
            const bool ok =
                __all_sync(0xffffffffu, mbar_wait_or_abort(acc_full0 + 8 * ab, u & 1, abort_flag, a.wait_cycles));
            if (!ok) {
                raise_abort(abort_flag, err, 4);
                break;
            }
            tc_fence_after();
            const uint32_t tbase = tmem + ((uint32_t)(32 * q4) << 16) + ab * a.acc_stride;
            int tx0, ty0;
            tile_of(P, item, tx0, ty0);
            const int py = ty0 + (m >> 4), px = tx0 + (m & 15);
            const TcWta r = tc_wta(tbase, (uint32_t)P.N, P.N, P.D, nullptr);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty0 + 8 * ab);
            if (py < P.H && px < P.W) {
                const size_t o = (size_t)py * P.W + px;
                if (P.disp_int) P.disp_int[o] = r.bidx;
                if (P.disp_sub) P.disp_sub[o] = tc_subpixel(r, P.D);
            }
        }
    } else if (warp == kTmaWarp) {
        // ================= TMA producer of guide tiles and cost rows ==========
        if (lane == 0) {
            uint32_t g = 0, gs = 0, gu = 0, t = 0, gpend = 0;   // gpend: guide tiles issued
            MemberView P, Q;   // the member of this tile and of the next one
            P.end = -1;
            P.index = 0;
            Q.end = -1;
            Q.index = 0;
            // guide tile of tile number tt (item `it` of member M) into slot
            // tt & 1, once the producers have released that slot; without
            // `block` only when it is already free.  Returns false on abort.
            auto issue_guide = [&](uint32_t tt, const MemberView& M, int it, bool block) -> bool {
                const uint32_t tb = tt & 1, u = tt >> 1;
                if (u > 0) {
                    if (!block) {
                        if (!mbar_try_wait(g_empty0 + 8 * tb, (u - 1) & 1)) return true;
                    } else if (!mbar_wait_or_abort(g_empty0 + 8 * tb, (u - 1) & 1, abort_flag, a.wait_cycles)) {
                        raise_abort(abort_flag, err, 7);
                        return false;
                    }
                }
                int gx0, gy0;
                tile_of(M, it, gx0, gy0);
                mbar_expect_tx(g_full0 + 8 * tb, (uint32_t)M.NH * M.KW * 8);
                tma_load_2d(smem_u32(g_base + tb * g_slot), &M.p->gmap, gx0 - M.rho8, gy0 - M.rho, g_full0 + 8 * tb);
                gpend = tt + 1;
                return true;
            };
            bool stop = false;
            for (int item = (int)blockIdx.x; item < a.nitems && !stop; item += grid, ++t) {
                if (item >= P.end) {
                    view_member(P, pairs, member_of(pairs, a.npairs, P.index, item));
                    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&P.p->tmap) : "memory");
                    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&P.p->gmap) : "memory");
                }
                int tx0, ty0;
                tile_of(P, item, tx0, ty0);
                const int xlo = tx0 - P.rho8;
                if (gpend == t && !issue_guide(t, P, item, true)) break;
                // the next tile's guide goes out as soon as its slot is free
                const int next = item + grid;
                const bool has_next = next < a.nitems;
                if (has_next && next >= Q.end) view_member(Q, pairs, member_of(pairs, a.npairs, Q.index, next));
                const uint32_t box = (uint32_t)P.R * (P.KW / 8) * P.Nb * 16;
                const int hr_lo = max(0, P.rho - ty0);
                const int hr_hi = min(P.NH, P.H - ty0 + P.rho);
                for (int h0 = hr_lo; h0 < hr_hi; h0 += P.R) {
                    const uint32_t s = gs, use = gu;
                    if (use > 0 && !mbar_wait_or_abort(empty0 + 8 * s, (use - 1) & 1, abort_flag, a.wait_cycles)) {
                        raise_abort(abort_flag, err, 2);
                        stop = true;
                        break;
                    }
                    mbar_expect_tx(full_b0 + 8 * s, box);
                    tma_load_4d(smem_u32(b_base + s * a.b_stage), &P.p->tmap, 0, 0, xlo >> 3, ty0 - P.rho + h0,
                                full_b0 + 8 * s);
                    ++g;
                    if (++gs == (uint32_t)S) {
                        gs = 0;
                        ++gu;
                    }
                    if (has_next && gpend == t + 1 && !issue_guide(t + 1, Q, next, false)) {
                        stop = true;
                        break;
                    }
                }
            }
            if (*abort_flag) {
                // let the copies still in flight land before the CTA exits
                const uint32_t n = g < (uint32_t)S ? g : (uint32_t)S;
                for (uint32_t x = g - n; x < g; ++x) mbar_wait(full_b0 + 8 * (x % S), (x / S) & 1);
                const uint32_t ng2 = gpend < 2 ? gpend : 2;
                for (uint32_t x = gpend - ng2; x < gpend; ++x) mbar_wait(g_full0 + 8 * (x & 1), (x >> 1) & 1);
            }
        }
    } else {
        // ================= MMA issuer =========================================
        if (lane == 0) {
            uint32_t gs = 0, gu = 0, t = 0;
            const uint64_t a_desc0 = sdesc(smem_u32(a_base), kALbo, 128);
            MemberView P;
            P.end = -1;
            P.index = 0;
            uint64_t b_desc0 = 0;
            uint32_t lbo_b = 0;
            bool stop = false;
            for (int item = (int)blockIdx.x; item < a.nitems && !stop; item += grid, ++t) {
                if (item >= P.end) {
                    view_member(P, pairs, member_of(pairs, a.npairs, P.index, item));
                    lbo_b = (uint32_t)P.Nb * 16;
                    b_desc0 = sdesc(smem_u32(b_base), lbo_b, 128);
                }
                const uint32_t ab = a.nacc == 2 ? (t & 1) : 0, u = a.nacc == 2 ? (t >> 1) : t;
                if (u > 0 && !mbar_wait_or_abort(acc_empty0 + 8 * ab, (u - 1) & 1, abort_flag, a.wait_cycles)) {
                    raise_abort(abort_flag, err, 5);
                    break;
                }
                tc_fence_after();
                const uint32_t dacc = tmem + ab * a.acc_stride;
                int tx0, ty0;
                tile_of(P, item, tx0, ty0);
                const int hr_lo = max(0, P.rho - ty0);
                const int hr_hi = min(P.NH, P.H - ty0 + P.rho);
                const int ksteps = P.KW / 16;
                const uint32_t idesc = P.idesc, idesc2 = P.idesc2;
                const bool split = P.split != 0;
                uint32_t accumulate = 0;
                for (int h0 = hr_lo; h0 < hr_hi; h0 += P.R) {
                    const int nr = min(P.R, hr_hi - h0);
                    const uint32_t s = gs, par = gu & 1;
                    if (!mbar_wait_or_abort(full_a0 + 8 * s, par, abort_flag, a.wait_cycles) ||
                        !mbar_wait_or_abort(full_b0 + 8 * s, par, abort_flag, a.wait_cycles)) {
                        raise_abort(abort_flag, err, 3);
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t ad = a_desc0 + ((s * a.a_stage) >> 4), bd = b_desc0 + ((s * a.b_stage) >> 4);
                    const int nk = nr * ksteps;
                    // the 14-bit address fields never carry into the descriptors'
                    // high words: few instructions per MMA for the issuing thread
                    const uint64_t ahi = ad & 0xffffffff00000000ull, bhi = bd & 0xffffffff00000000ull;
                    uint32_t alo = (uint32_t)ad, blo = (uint32_t)bd;
                    const uint32_t astep = (2 * kALbo) >> 4, bstep = (2 * lbo_b) >> 4;
                    if (!split) {
                        umma_f16(dacc, ahi | alo, bhi | blo, idesc, accumulate);
#pragma unroll 4
                        for (int k = 1; k < nk; ++k) {
                            alo += astep;
                            blo += bstep;
                            umma_f16(dacc, ahi | alo, bhi | blo, idesc, 1u);
                        }
                    } else {
                        // B rows 0..127 into columns 0..127, rows 128..Nb-1 (with the
                        // ones row) into columns 128..Nb-1
                        const uint32_t b2 = (128 * 16) >> 4;
                        for (int k = 0; k < nk; ++k) {
                            umma_f16(dacc, ahi | alo, bhi | blo, idesc, accumulate);
                            umma_f16(dacc + 128, ahi | alo, bhi | (blo + b2), idesc2, accumulate);
                            accumulate = 1;
                            alo += astep;
                            blo += bstep;
                        }
                    }
                    accumulate = 1;
                    umma_commit(empty0 + 8 * s);
                    if (++gs == (uint32_t)S) {
                        gs = 0;
                        ++gu;
                    }
                }
                if (stop) break;
                umma_commit(acc_full0 + 8 * ab);
            }
            umma_commit(drain_bar);
            mbar_wait(drain_bar, 0);
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, a.tmem_cols);
}

}  // namespace
}  // namespace fbs

namespace fbs {

size_t tc_batch_table_bytes(int n) { return sizeof(TcBatchPair) * (size_t)(n > 0 ? n : 0); }

cudaError_t tc_batch_prepare(int n, const TcBatchMember* m, bool bf16, void* host_table, TcBatchLaunch* out)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    if (n < 1 || !m || !host_table || !out) return cudaErrorInvalidValue;
    struct Geo {
        int N, Nb, split, rho8, KW, NH, ntx, ntiles, variant;
        uint32_t a_row, b_row;
        double tile_work;
    };
    std::vector<Geo> g(n);
    for (int i = 0; i < n; ++i) {
        const TcBatchMember& q = m[i];
        if (q.D < 1 || q.D > 256 || q.radius < 0 || q.radius > 24 || q.H < 1 || q.W < 1) return cudaErrorInvalidValue;
        Geo& e = g[i];
        e.N = round_up(q.D, 16);
        e.Nb = tc_block_rows(q.D);
        e.split = e.Nb > 256 ? 1 : 0;
        e.rho8 = round_up(q.radius, 8);
        e.KW = round_up(16 + e.rho8 + q.radius, 16);
        e.NH = kTH + 2 * q.radius;
        e.ntx = (q.W + kTW - 1) / kTW;
        e.ntiles = e.ntx * ((q.H + kTH - 1) / kTH);
        e.variant = batch_variant(q.radius);
        e.a_row = (uint32_t)(e.KW / 8) * kALbo;
        e.b_row = (uint32_t)(e.KW / 8) * e.Nb * 16;
        // a tile: NH window rows of KW weight columns, each feeding an MMA of N = Nb
        e.tile_work = (double)e.NH * e.KW * (e.Nb + 64);
    }
    // table order: by variant, then largest tiles first
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return g[x].variant != g[y].variant ? g[x].variant < g[y].variant : g[x].tile_work > g[y].tile_work;
    });
    std::vector<TcBatchPair> t(n);
    const double log2e = 1.4426950408889634;
    TcBatchLaunch& l = *out;
    l.ngroups = 0;
    for (int k0 = 0; k0 < n;) {
        const int v = g[order[k0]].variant;
        int k1 = k0;
        while (k1 < n && g[order[k1]].variant == v) ++k1;
        // the group's stage layout: the largest R (<= kMaxR) whose stages of R
        // rows of its largest member fit at least twice in 227 KB, then as many
        // stages (<= 6) as fit
        int kw_max = 0, nh_max = 0;
        uint32_t a_max = 0, b_max = 0, acc_stride = 0;
        for (int k = k0; k < k1; ++k) {
            const Geo& e = g[order[k]];
            kw_max = std::max(kw_max, e.KW);
            nh_max = std::max(nh_max, e.NH);
            a_max = std::max(a_max, e.a_row);
            b_max = std::max(b_max, e.b_row);
            acc_stride = std::max(acc_stride, (uint32_t)e.N + 16);
        }
        int R = 0, S = 0;
        BatchSmem L{};
        for (int r = kMaxR; r >= 1 && !R; --r)
            for (int s = 6; s >= 2; --s) {
                L = batch_smem_layout(s, (uint32_t)r * a_max, (uint32_t)r * b_max, kw_max, nh_max);
                if (L.total <= 227 * 1024) {
                    R = r;
                    S = s;
                    break;
                }
            }
        if (!R) return cudaErrorInvalidValue;
        const uint32_t a_stage = (uint32_t)R * a_max, b_stage = (uint32_t)R * b_max;
        int items = 0;
        for (int k = k0; k < k1; ++k) {
            const TcBatchMember& q = m[order[k]];
            const Geo& e = g[order[k]];
            TcBatchPair& b = t[k];
            b.H = q.H;
            b.W = q.W;
            b.D = q.D;
            b.N = e.N;
            b.Nb = e.Nb;
            b.split = e.split;
            b.rho = q.radius;
            b.rho8 = e.rho8;
            b.KW = e.KW;
            b.NH = e.NH;
            b.ntx = e.ntx;
            // window rows per stage: as many as the group's stage sizes hold
            b.R = (int)std::min<uint32_t>((uint32_t)kMaxR, std::min(a_stage / e.a_row, b_stage / e.b_row));
            b.variant = v;
            b.item0 = items;
            b.items = e.ntiles;
            items += e.ntiles;
            b.neg_ks = (float)(-log2e / ((double)q.sigma_s * q.sigma_s));
            b.neg_kr = (float)(-log2e / ((double)q.sigma_r * q.sigma_r));
            b.idesc = tc_idesc(bf16, e.split ? 128 : e.Nb);
            b.idesc2 = tc_idesc(bf16, e.split ? e.Nb - 128 : 16);
            b.disp_int = q.disp_int;
            b.disp_sub = q.disp_sub;
            if (encode_cost_map(enc, &b.tmap, q.cost, q.H, q.W, e.Nb, e.KW, b.R, bf16) != CUDA_SUCCESS ||
                encode_guide_map(enc, &b.gmap, q.rgbx, q.H, q.W, rgbx_pitch(q.W), e.KW, e.NH) != CUDA_SUCCESS)
                return cudaErrorInvalidValue;
        }
        TcBatchGroup& G = l.group[l.ngroups++];
        G.variant = v;
        G.first = k0;
        G.npairs = k1 - k0;
        G.nitems = items;
        G.R = R;
        G.S = S;
        G.nacc = 2 * acc_stride <= 512 ? 2 : 1;
        G.kw_max = kw_max;
        G.nh_max = nh_max;
        G.a_stage = a_stage;
        G.b_stage = b_stage;
        G.acc_stride = acc_stride;
        uint32_t cols = 32;
        while (cols < (uint32_t)G.nacc * acc_stride) cols <<= 1;
        G.tmem_cols = cols;
        G.smem = L.total;
        k0 = k1;
    }
    memcpy(host_table, t.data(), tc_batch_table_bytes(n));
    return cudaSuccess;
}

namespace {

typedef void (*BatchKernel)(TcBatchArgs, int*);

// The kernel instance of producer variant v (see batch_variant).
template <bool BF16>
BatchKernel batch_kernel(int v)
{
    static const BatchKernel k[] = {
        aggregate_tc_batch_kernel<BF16, 1, 0>,  aggregate_tc_batch_kernel<BF16, 1, 1>,
        aggregate_tc_batch_kernel<BF16, 2, 0>,  aggregate_tc_batch_kernel<BF16, 2, 1>,
        aggregate_tc_batch_kernel<BF16, 3, 0>,  aggregate_tc_batch_kernel<BF16, 3, 1>,
        aggregate_tc_batch_kernel<BF16, 4, 0>,  aggregate_tc_batch_kernel<BF16, 4, 1>,
        aggregate_tc_batch_kernel<BF16, 5, 0>,  aggregate_tc_batch_kernel<BF16, 5, 1>,
        aggregate_tc_batch_kernel<BF16, 6, 0>,  aggregate_tc_batch_kernel<BF16, 6, 1>,
        aggregate_tc_batch_kernel<BF16, 7, 0>,  aggregate_tc_batch_kernel<BF16, 7, 1>,
        aggregate_tc_batch_kernel<BF16, 8, 0>,  aggregate_tc_batch_kernel<BF16, 8, 1>,
        aggregate_tc_batch_kernel<BF16, 10, 2>, aggregate_tc_batch_kernel<BF16, 13, 2>};
    return v >= 0 && v < (int)(sizeof(k) / sizeof(k[0])) ? k[v] : nullptr;
}

}  // namespace

cudaError_t launch_aggregate_tc_batch(const void* dev_table, const TcBatchLaunch& l, bool bf16, int* err,
                                      int num_sms, long long wait_cycles, cudaStream_t stream)
{
    if (!dev_table || l.ngroups < 1) return cudaErrorInvalidValue;
    for (int i = 0; i < l.ngroups; ++i) {
        const TcBatchGroup& G = l.group[i];
        BatchKernel k = bf16 ? batch_kernel<true>(G.variant) : batch_kernel<false>(G.variant);
        if (!k || G.nitems < 1) return cudaErrorInvalidValue;
        TcBatchArgs a;
        a.pairs = (const TcBatchPair*)dev_table + G.first;
        a.npairs = G.npairs;
        a.nitems = G.nitems;
        a.S = G.S;
        a.nacc = G.nacc;
        a.kw_max = G.kw_max;
        a.nh_max = G.nh_max;
        a.a_stage = G.a_stage;
        a.b_stage = G.b_stage;
        a.acc_stride = G.acc_stride;
        a.tmem_cols = G.tmem_cols;
        a.wait_cycles = wait_cycles > 0 ? wait_cycles : kWaitCycles;
        cudaError_t e = raise_smem_limit((const void*)k, G.smem);
        if (e != cudaSuccess) return e;
        const int grid = G.nitems < num_sms ? G.nitems : num_sms;
        fbs::note_launch();
        k<<<grid, kThreads, G.smem, stream>>>(a, err);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace fbs
