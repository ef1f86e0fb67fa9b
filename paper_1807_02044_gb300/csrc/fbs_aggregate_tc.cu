// Steps 2-4 of fast bilateral stereo on the 5th-generation tensor cores.
//
// Eq. (6) for a tile of M = 128 pixels (16 x 8) is a product
//     Agg[m][d] * den[m] = sum_k  W[m][k] * C[k][d],
// where k runs over the window pixels the tile can reach, W[m][k] is the
// bilateral weight of Eq. (7)-(8) (zero outside pixel m's window) and
// C[k][d] the cost volume.  The K dimension is walked one window row at a
// time: for window row hr the CTA
//   * loads C[row hr, KW columns][Nb rows] with TMA from the 16-bit x-blocked
//     cost volume [H][W/8][Nb][8] (B operand, K-major; Nb = round_up(D,16) + 16
//     rows per block: the costs, zero rows up to round_up(D,16), a row of ones
//     and 15 zero rows): one box per block of 8 columns, each a contiguous
//     Nb x 16-byte block that lands as Nb/8 core matrices; out-of-image columns
//     and rows are zero-filled;
//   * computes the weights of every tile pixel whose window contains row hr
//     (A operand, K-major, 128 rows x KW columns) into shared memory: each
//     weight is one exp2 in FP32, rounded to BF16 or FP16;
//   * issues KW/16 tcgen05.mma (kind::f16, M=128, N=Nb, K=16; two of N = 128
//     and Nb - 128 when Nb > 256) accumulating in FP32 in tensor memory.  The
//     ones row makes the same product also sum the rounded weights, so the
//     numerator and the normaliser use the same weights.
// A ring of S stages of R rows each (S >= 2) lets the threads produce the
// next stage while the tensor core works on the current one; TMA runs ahead.  After the last row,
// four warps read the accumulator rows (one pixel per TMEM lane), normalise
// in FP32, and do WTA (smallest d on ties) and Eq. (10) in registers.
//
// Shared-memory operand layout (no swizzle, canonical K-major core matrices
// of 8 rows x 16 bytes): element (row r, k) of an operand sits at
//     (k / 8) * LBO + r * 16 + (k % 8) * 2,
// i.e. the stride between core matrices along the rows (SBO) is 128 bytes and
// along K (LBO) 16 bytes per row plus padding: 128 * 16 + 64 for the weights
// (the padding spreads the producers' stores over the banks), Nb * 16 for the
// costs.  TMA writes a box of 8 columns x Nb disparities in exactly that order,
// so B needs no rearrangement.  All operands live in
// shared memory; warp roles and mbarrier pipelines are described at the kernel.
//
// Every wait on an mbarrier is bounded (iteration and clock limits); on a
// timeout the kernel records an error code, stops issuing work, drains what
// it issued, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fbs_internal.cuh"
#include "tc_aggregate.cuh"

namespace fbs {
namespace {

using namespace tca;

struct TcParams {
    int H, W, C, D;
    int N;          // round_up(D, 16): disparity rows
    int Nb;         // rows of a B stage: N, plus 16 normaliser rows (the ones row and 15 zero rows)
    int split;      // Nb > 256: two MMAs per K-step, B rows 0..127 and 128..Nb-1
    int rho, rho8, KW, NH, ntx, ntiles;
    int R;          // window rows per pipeline stage
    int S;          // pipeline stages (weights and cost rows share the stage index)
    int nacc;       // accumulator buffers in TMEM (2 = epilogue overlaps the next tile)
    uint32_t acc_stride, den_col, tmem_cols;
    float neg_ks, neg_kr;
    uint32_t idesc, idesc2;   // the (first) MMA's instruction descriptor; the second MMA's when split
    long long wait_cycles;   // limit of one pipeline wait (on another role's progress)
};

struct TcSmem {
    size_t a_off, b_off, g_off, bar_off, misc_off, sy_off, total;
};

// Per stage: R window rows of weights (A, (KW/8) x kALbo bytes each) and R
// rows of costs (B, (KW/8) x Nb x 16 bytes each).
__host__ __device__ inline TcSmem tc_smem_layout(int KW, int Nb, int NH, int R, int S)
{
    TcSmem s;
    size_t o = 0;
    s.a_off = o;
    o += (size_t)S * R * (KW / 8) * kALbo;
    s.b_off = o;
    o += (size_t)S * R * (KW / 8) * Nb * 16;
    o = (o + 127) & ~(size_t)127;
    s.g_off = o;
    o += (size_t)2 * NH * KW * 8;
    o = (o + 15) & ~(size_t)15;
    s.bar_off = o;
    o += (size_t)(3 * S + 9) * 8;
    s.misc_off = o;
    o += 16;
    s.sy_off = o;         // spatial y-terms, one packed pair per row offset
    o += (size_t)kMaxRho2 * 8;
    s.total = o + 1024;   // slack for aligning the base to 1024 bytes
    return s;
}

// The persistent tile walk of a CTA (tiles blockIdx.x, + gridDim.x, ...) with
// the tile's column and row carried incrementally (no division per tile).
struct TileWalk {
    int tile, tx, ty, dx, dy, ntx;
    __device__ __forceinline__ TileWalk(int ntx_)
        : tile((int)blockIdx.x), tx((int)blockIdx.x % ntx_), ty((int)blockIdx.x / ntx_),
          dx((int)gridDim.x % ntx_), dy((int)gridDim.x / ntx_), ntx(ntx_) {}
    __device__ __forceinline__ void next()
    {
        tile += (int)gridDim.x;
        tx += dx;
        ty += dy;
        if (tx >= ntx) {
            tx -= ntx;
            ++ty;
        }
    }
};

// Warp roles: 0-15 weight producers, 16-19 epilogue (TMEM lane quarters 0-3),
// 20 TMA producer (guide tiles and cost rows), 21 MMA issuer.  NPT = column
// pairs per pixel and window row of one producer thread (ceil((rho + 1) / 2),
// rounded up to an instantiated count).
//
// Pipeline: a stage holds R consecutive window rows of one tile (the last
// stage of a tile may hold fewer).  For stage g in slot s = g % S:
//   producers  wait empty[s] (stage g - S consumed), write R rows of weights,
//              arrive full_a[s] (one arrival per warp);
//   TMA        waits empty[s], loads R cost rows, full_b[s] completes on bytes;
//   MMA        waits full_a[s] and full_b[s], issues R * KW/16 MMAs, commits
//              to empty[s]; after a tile's last stage commits acc_full[ab];
//   epilogue   waits acc_full[ab], reads the accumulator, arrives acc_empty[ab].
// One wait/commit pair per R rows keeps the single-thread control path
// (which shares its scheduler with busy warps) off the critical path.
template <bool BF16, int NPT, int PM>
__global__ void __launch_bounds__(kThreads, 1)
aggregate_tc_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap gmap, TcParams p,
                    float* __restrict__ agg_out, int32_t* __restrict__ disp_int, float* __restrict__ disp_sub,
                    int* __restrict__ err)
{
    extern __shared__ uint8_t smem_raw[];
    // align by an offset from the __shared__ array itself (not an integer round
    // trip), so the compiler keeps every operand access a 32-bit shared one
    uint8_t* sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const TcSmem L = tc_smem_layout(p.KW, p.Nb, p.NH, p.R, p.S);
    uint8_t* a_base = sm + L.a_off;
    uint8_t* b_base = sm + L.b_off;
    uint2* gtile = (uint2*)(sm + L.g_off);   // [2][NH][KW] of (RGBX, |colour|^2)
    const uint32_t bars = smem_u32(sm + L.bar_off);
    const uint32_t full_a0 = bars, full_b0 = bars + 8 * p.S, empty0 = bars + 16 * p.S,
                   acc_full0 = bars + 24 * p.S, acc_empty0 = acc_full0 + 16, drain_bar = acc_empty0 + 16,
                   g_full0 = drain_bar + 8, g_empty0 = g_full0 + 16;
    uint32_t* misc = (uint32_t*)(sm + L.misc_off);   // [0] TMEM base, [1] abort flag
    volatile uint32_t* abort_flag = misc + 1;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int KW = p.KW, R = p.R, S = p.S;
    const uint32_t a_row = (uint32_t)(KW / 8) * kALbo;      // bytes of one window row of weights
    const uint32_t lbo_b = (uint32_t)p.Nb * 16;
    const uint32_t b_row = (uint32_t)(KW / 8) * lbo_b;      // bytes of one window row of costs
    const uint32_t a_stage = a_row * R, b_stage = b_row * R;

    // ---- set-up --------------------------------------------------------------
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full_a0 + 8 * s, kProducerWarps);   // one elected arrival per producer warp
            mbar_init(full_b0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(acc_full0 + 8 * s, 1);
            mbar_init(acc_empty0 + 8 * s, kEpilogue / 32);   // one per epilogue warp
            mbar_init(g_full0 + 8 * s, 1);
            mbar_init(g_empty0 + 8 * s, kProducerWarps);
        }
        mbar_init(drain_bar, 1);
        misc[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmap) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&gmap) : "memory");
    }
    if (warp == 0) tmem_alloc(smem_u32(&misc[0]), p.tmem_cols);
    // spatial y-term of row offset dy, (ks dy^2, ks dy^2), at index dy + rho
    uint64_t* sytab = (uint64_t*)(sm + L.sy_off);
    for (int i = tid; i <= 2 * p.rho; i += kThreads) {
        const int dy = i - p.rho;
        const float sy = (float)(dy * dy) * p.neg_ks;
        sytab[i] = f2_pack(sy, sy);
    }
    for (int i = tid; i < (int)(S * a_stage / 16); i += kThreads) ((uint4*)a_base)[i] = make_uint4(0, 0, 0, 0);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = misc[0];
    // With a programmatic launch the set-up above overlaps the end of the
    // kernel that writes the cost volume and the guide; everything below reads
    // them, so every thread waits here until that kernel has completed and its
    // writes are visible (a no-op for an ordinary launch).
    asm volatile("griddepcontrol.wait;" ::: "memory");

    if (warp < kProducerWarps) {
        // ================= weight producers =================================
        // Warp w covers the pixel rows ty = 2 (w >> 2) and ty + 1 of the tile
        // and, within every stage, the window rows r with r % 4 == w % 4; lane
        // -> pixel column xm = lane & 15 and pair phase h = lane >> 4.  Pixel
        // (xm, y) needs window columns kcen - rho .. kcen + rho (kcen = xm +
        // rho8), covered by rho + 1 pairs of adjacent columns (k, k + 1)
        // starting at the even column c0 <= kcen - rho; the thread computes the
        // pairs 2 j + h (j < NPT) of both pixels of its column, which share
        // every guide load (the same window position q).  Columns a pixel never
        // reaches are never written and stay zero.  Whether a window row lies
        // inside a pixel row's window is uniform over the warp, and the row is
        // computed only for the pixel rows whose window it lies in (zeros for
        // the other).  PM says which pairs exist: all NPT (odd radius), all
        // but the last one of phase 1 (even radius), or per-pair flags.
        // Colour distance: |q - p|^2 = |q|^2 + |p|^2 - 2 q.p, exact in integers
        // (|q|^2 comes with the guide tile, q.p is one dp4a).  It is below 2^23,
        // so carrying kMagic in |p|^2 turns the integer into the bits of
        // 2^23 + c and one packed subtraction gives both columns' c as exact
        // floats; the exponent argument c*neg_kr + (sx + sy) of a column pair is
        // one packed add and one packed FMA (the same roundings as scalar code).
        const int ty = 2 * (warp >> 2), rq = warp & 3;
        const int xm = lane & 15, h = lane >> 4;
        const int m0 = 16 * ty + xm;   // A row of the upper pixel; the lower one is m0 + 16
        const int kcen = xm + p.rho8;
        const int c0 = (kcen - p.rho) & ~1;
        const int np = p.rho + 1;
        // pair j of the thread: columns k, k + 1 with k = c0 + 2 h + 4 j, guide
        // entries at byte 8 (c0 + 2 h) + 32 j of a guide row
        bool on[NPT];
#pragma unroll
        for (int j = 0; j < NPT; ++j)
            on[j] = PM == 0 ? true : PM == 1 ? (j < NPT - 1 || h == 0) : 2 * j + h < np;
        const TcPairOffsets po = tc_pair_offsets(c0 + 2 * h, m0);
        const uint32_t gcol = (uint32_t)(c0 + 2 * h) * 8;   // byte offset of pair 0 in a guide row
        const uint32_t g_row = (uint32_t)KW * 8;            // bytes of one guide row
        const float ninf = __int_as_float(0xff800000);
        const uint64_t magic2 = f2_pack(-8388608.f, -8388608.f);
        const uint64_t nkr2 = f2_pack(p.neg_kr, p.neg_kr);
        const unsigned two_rho = (unsigned)(2 * p.rho);
        uint32_t gs = 0, gu = 0, t = 0;   // stage slot and use count of the next stage
        bool stop = false;
        for (TileWalk tw(p.ntx); tw.tile < p.ntiles && !stop; tw.next(), ++t) {
            const int tx0 = tw.tx * kTW, ty0 = tw.ty * kTH;
            const int xlo = tx0 - p.rho8;
            const uint32_t tb = t & 1;
            if (!mbar_wait_or_abort(g_full0 + 8 * tb, (t >> 1) & 1, abort_flag, p.wait_cycles)) {
                raise_abort(abort_flag, err, 6);
                break;
            }
            const uint8_t* gt = (const uint8_t*)(gtile + tb * (p.NH * KW));
            // the two pixels' colours and, per pair, the spatial x-terms, or -inf
            // when the column is outside the window or the image (pixels outside
            // the image only feed their own accumulator rows, never stored)
            const uint2 pc0 = *(const uint2*)(gt + (ty + p.rho) * g_row + kcen * 8);
            const uint2 pc1 = *(const uint2*)(gt + (ty + 1 + p.rho) * g_row + kcen * 8);
            const uint32_t pcol0 = pc0.x, pp0 = pc0.y + kMagic, pcol1 = pc1.x, pp1 = pc1.y + kMagic;
            uint64_t sxp[NPT];
#pragma unroll
            for (int j = 0; j < NPT; ++j) {
                const int k = c0 + 2 * h + 4 * j;
                const int d0 = k - kcen, d1 = d0 + 1;
                const int x0 = xlo + k;
                const float s0 = (d0 >= -p.rho && d0 <= p.rho && (unsigned)x0 < (unsigned)p.W)
                                     ? (float)(d0 * d0) * p.neg_ks : ninf;
                const float s1 = (d1 >= -p.rho && d1 <= p.rho && (unsigned)(x0 + 1) < (unsigned)p.W)
                                     ? (float)(d1 * d1) * p.neg_ks : ninf;
                sxp[j] = f2_pack(s0, s1);
            }
            const uint8_t* gth = gt + gcol;
            auto row_pairs = [&](uint8_t* arow, const uint8_t* grow, uint64_t sy0, uint64_t sy1, int which)
                                 __attribute__((always_inline)) {
                tc_row_pairs<BF16, NPT>(arow, grow, po, on, sxp, sy0, sy1, which, pcol0, pp0, pcol1, pp1, magic2,
                                        nkr2);
            };
            const int hr_lo = max(0, p.rho - ty0);
            const int hr_hi = min(p.NH, p.H - ty0 + p.rho);
            for (int h0 = hr_lo; h0 < hr_hi; h0 += R) {
                const int nr = min(R, hr_hi - h0);
                const uint32_t s = gs, use = gu;   // g % S, g / S, carried below
                // one lane waits for the MMAs that last read stage s; the warp follows
                bool ok = true;
                if (lane == 0 && use > 0) ok = mbar_wait_or_abort(empty0 + 8 * s, (use - 1) & 1, abort_flag, p.wait_cycles);
                if (!__shfl_sync(0xffffffffu, ok, 0)) {
                    raise_abort(abort_flag, err, 1);
                    stop = true;
                    break;
                }
                uint8_t* ast = a_base + s * a_stage;
#pragma unroll
                for (int r = rq; r < kMaxR; r += 4) {
                    if (r >= nr) break;
                    const int hr = h0 + r;
                    const int dy = hr - ty;   // row offset + rho of the upper pixel
                    const bool in0 = (unsigned)dy <= two_rho, in1 = (unsigned)(dy - 1) <= two_rho;
                    uint8_t* arow = ast + r * a_row;
                    const uint8_t* grow = gth + hr * g_row;
                    // uniform over the warp: both pixel rows, one of them, or neither
                    if (in0 && in1)
                        row_pairs(arow, grow, sytab[dy], sytab[dy - 1], 3);
                    else if (in0)
                        row_pairs(arow, grow, sytab[dy], 0ull, 1);
                    else if (in1)
                        row_pairs(arow, grow, 0ull, sytab[dy - 1], 2);
                    else
                        row_pairs(arow, grow, 0ull, 0ull, 0);
                }
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive(full_a0 + 8 * s);
                if (++gs == (uint32_t)S) {
                    gs = 0;
                    ++gu;
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(g_empty0 + 8 * tb);   // this tile's guide is no longer read
        }
    } else if (warp < kTmaWarp) {
        // ================= epilogue: TMEM -> normalise -> WTA -> Eq. (10) ======
        const int q4 = warp - kEpiWarp0;    // TMEM lane quarter
        const int m = 32 * q4 + lane;       // pixel of the tile == TMEM lane
        uint32_t t = 0;
        for (TileWalk tw(p.ntx); tw.tile < p.ntiles; tw.next(), ++t) {
            const uint32_t ab = p.nacc == 2 ? (t & 1) : 0, u = p.nacc == 2 ? (t >> 1) : t;
            // tcgen05.ld is warp-collective: the whole warp continues or stops
            const bool ok = __all_sync(0xffffffffu, mbar_wait_or_abort(acc_full0 + 8 * ab, u & 1, abort_flag, p.wait_cycles));
            if (!ok) {
                raise_abort(abort_flag, err, 4);
                break;
            }
            tc_fence_after();
            const uint32_t tbase = tmem + ((uint32_t)(32 * q4) << 16) + ab * p.acc_stride;
            const int tx0 = tw.tx * kTW, ty0 = tw.ty * kTH;
            const int py = ty0 + (m >> 4), px = tx0 + (m & 15);
            const bool pvalid = py < p.H && px < p.W;
            float* arow = (agg_out && pvalid) ? agg_out + ((size_t)py * p.W + px) * p.D : nullptr;
            const TcWta r = tc_wta(tbase, p.den_col, p.N, p.D, arow);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty0 + 8 * ab);
            if (pvalid) {
                const size_t o = (size_t)py * p.W + px;
                if (disp_int) disp_int[o] = r.bidx;
                if (disp_sub) disp_sub[o] = tc_subpixel(r, p.D);
            }
        }
    } else if (warp == kTmaWarp) {
        // ================= TMA producer of guide tiles and cost rows ==========
        if (lane == 0) {
            uint32_t g = 0, gs = 0, gu = 0, t = 0, gpend = 0;   // gpend: guide tiles issued
            const uint32_t guide_bytes = (uint32_t)p.NH * KW * 8;
            // guide tile of tile number tt at (tx0, ty0) into slot tt & 1, once the
            // producers have released that slot (tile tt - 2); without `block`
            // only when the slot is already free.  Returns false on abort.
            auto issue_guide = [&](uint32_t tt, int tx0, int ty0, bool block) -> bool {
                const uint32_t tb = tt & 1, u = tt >> 1;
                if (u > 0) {
                    if (!block) {
                        if (!mbar_try_wait(g_empty0 + 8 * tb, (u - 1) & 1)) return true;
                    } else if (!mbar_wait_or_abort(g_empty0 + 8 * tb, (u - 1) & 1, abort_flag, p.wait_cycles)) {
                        raise_abort(abort_flag, err, 7);
                        return false;
                    }
                }
                mbar_expect_tx(g_full0 + 8 * tb, guide_bytes);
                tma_load_2d(smem_u32(gtile + tb * (p.NH * KW)), &gmap, tx0 - p.rho8, ty0 - p.rho, g_full0 + 8 * tb);
                gpend = tt + 1;
                return true;
            };
            bool stop = false;
            for (TileWalk tw(p.ntx); tw.tile < p.ntiles && !stop; tw.next(), ++t) {
                const int tx0 = tw.tx * kTW, ty0 = tw.ty * kTH;
                const int xlo = tx0 - p.rho8;
                if (gpend == t && !issue_guide(t, tx0, ty0, true)) break;
                // the next tile's guide goes out as soon as its slot is free,
                // between this tile's cost rows, so that it has landed when the
                // producers reach that tile
                TileWalk nx = tw;
                nx.next();
                const bool has_next = nx.tile < p.ntiles;
                const int hr_lo = max(0, p.rho - ty0);
                const int hr_hi = min(p.NH, p.H - ty0 + p.rho);
                for (int h0 = hr_lo; h0 < hr_hi; h0 += R) {
                    const uint32_t s = gs, use = gu;   // g % S, g / S
                    if (use > 0 && !mbar_wait_or_abort(empty0 + 8 * s, (use - 1) & 1, abort_flag, p.wait_cycles)) {
                        raise_abort(abort_flag, err, 2);
                        stop = true;
                        break;
                    }
                    // one box: 8 columns x Nb rows x KW/8 blocks x R window rows
                    mbar_expect_tx(full_b0 + 8 * s, b_stage);
                    tma_load_4d(smem_u32(b_base + s * b_stage), &tmap, 0, 0, xlo >> 3, ty0 - p.rho + h0, full_b0 + 8 * s);
                    ++g;
                    if (++gs == (uint32_t)S) {
                        gs = 0;
                        ++gu;
                    }
                    if (has_next && gpend == t + 1 && !issue_guide(t + 1, nx.tx * kTW, nx.ty * kTH, false)) {
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
            uint32_t gs = 0, gu = 0, t = 0;   // stage slot and use count
            // descriptors of stage 0, row 0, K-step 0; other positions add their
            // byte offset >> 4 to the 14-bit start-address field
            const uint64_t a_desc0 = sdesc(smem_u32(a_base), kALbo, 128);
            const uint64_t b_desc0 = sdesc(smem_u32(b_base), lbo_b, 128);
            bool stop = false;
            for (TileWalk tw(p.ntx); tw.tile < p.ntiles && !stop; tw.next(), ++t) {
                const uint32_t ab = p.nacc == 2 ? (t & 1) : 0, u = p.nacc == 2 ? (t >> 1) : t;
                if (u > 0 && !mbar_wait_or_abort(acc_empty0 + 8 * ab, (u - 1) & 1, abort_flag, p.wait_cycles)) {
                    raise_abort(abort_flag, err, 5);
                    break;
                }
                tc_fence_after();
                const uint32_t dacc = tmem + ab * p.acc_stride;
                const int ty0 = tw.ty * kTH;
                const int hr_lo = max(0, p.rho - ty0);
                const int hr_hi = min(p.NH, p.H - ty0 + p.rho);
                uint32_t accumulate = 0;
                for (int h0 = hr_lo; h0 < hr_hi; h0 += R) {
                    const int nr = min(R, hr_hi - h0);
                    const uint32_t s = gs, par = gu & 1;   // g % S, (g / S) & 1
                    if (!mbar_wait_or_abort(full_a0 + 8 * s, par, abort_flag, p.wait_cycles) ||
                        !mbar_wait_or_abort(full_b0 + 8 * s, par, abort_flag, p.wait_cycles)) {
                        raise_abort(abort_flag, err, 3);
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    // K steps of 16 walk a stage's rows contiguously: a row is KW/16
                    // steps of 2 core-matrix columns in both operands
                    uint64_t ad = a_desc0 + ((s * a_stage) >> 4), bd = b_desc0 + ((s * b_stage) >> 4);
                    const int nk = nr * (KW / 16);
                    // the 14-bit address fields never carry into the descriptors'
                    // high words: few instructions per MMA for the issuing thread,
                    // which shares its scheduler with five busy warps
                    const uint64_t ahi = ad & 0xffffffff00000000ull, bhi = bd & 0xffffffff00000000ull;
                    uint32_t alo = (uint32_t)ad, blo = (uint32_t)bd;
                    const uint32_t astep = (2 * kALbo) >> 4, bstep = (2 * lbo_b) >> 4;
                    if (!p.split) {
                        umma_f16(dacc, ahi | alo, bhi | blo, p.idesc, accumulate);
                        accumulate = 1;
#pragma unroll 4
                        for (int k = 1; k < nk; ++k) {
                            alo += astep;
                            blo += bstep;
                            umma_f16(dacc, ahi | alo, bhi | blo, p.idesc, 1u);
                        }
                    } else {
                        // B rows 0..127 into accumulator columns 0..127, rows
                        // 128..Nb-1 (with the ones row) into columns 128..Nb-1:
                        // an MMA of N <= 128 costs the same ~88 cycles as one of
                        // N = 16, so 128 + 144 beats 256 + a separate 16
                        const uint32_t b2 = (128 * 16) >> 4;
                        for (int k = 0; k < nk; ++k) {
                            umma_f16(dacc, ahi | alo, bhi | blo, p.idesc, accumulate);
                            umma_f16(dacc + 128, ahi | alo, bhi | (blo + b2), p.idesc2, accumulate);
                            accumulate = 1;
                            alo += astep;
                            blo += bstep;
                        }
                    }
                    umma_commit(empty0 + 8 * s);
                    if (++gs == (uint32_t)S) {
                        gs = 0;
                        ++gu;
                    }
                }
                if (stop) break;
                umma_commit(acc_full0 + 8 * ab);
            }
            // every MMA issued by this thread has completed before the CTA exits
            umma_commit(drain_bar);
            mbar_wait(drain_bar, 0);
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, p.tmem_cols);
}

template <bool BF16>
__global__ void hwd_to_xblock16_kernel(const float* __restrict__ in, int H, int W, int D,
                                       typename Op16<BF16>::T* __restrict__ out)
{
    // one thread per (row, block of 8 columns, disparity): 8 values, 16 bytes out
    const int nxb = (W + 7) / 8;
    const int dp = tc_block_rows(D);
    const size_t n = (size_t)H * nxb * D;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int d = (int)(i % D);
        const size_t yb = i / D;
        const int xb = (int)(yb % nxb), y = (int)(yb / nxb);
        typename Op16<BF16>::T v[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int x = 8 * xb + c;
            v[c] = Op16<BF16>::from(x < W ? in[((size_t)y * W + x) * D + d] : 0.f);
        }
        uint32_t w[4];
#pragma unroll
        for (int c = 0; c < 4; ++c)
            w[c] = (uint32_t)*reinterpret_cast<const unsigned short*>(&v[2 * c]) |
                   ((uint32_t)*reinterpret_cast<const unsigned short*>(&v[2 * c + 1]) << 16);
        *reinterpret_cast<uint4*>(out + (yb * dp + d) * 8) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

template <bool BF16>
__global__ void xblock16_pad_kernel(int H, int W, int D, typename Op16<BF16>::T* __restrict__ out)
{
    // rows D .. Dp-1 of every block: zero, except row round_up(D,16) = all ones
    const int nxb = (W + 7) / 8;
    const int n16 = (D + 15) / 16 * 16, dp = tc_block_rows(D), extra = dp - D;
    const uint16_t one = BF16 ? (uint16_t)0x3F80 : (uint16_t)0x3C00;
    const size_t n = (size_t)H * nxb * extra;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int d = D + (int)(i % extra);
        const size_t yb = i / extra;
        const uint32_t v = (d == n16 && dp > n16) ? ((uint32_t)one | ((uint32_t)one << 16)) : 0u;
        *reinterpret_cast<uint4*>(out + (yb * dp + d) * 8) = make_uint4(v, v, v, v);
    }
}

}  // namespace

cudaError_t launch_hwd_to_xblock16(const float* in, int H, int W, int D, bool bf16, void* out, cudaStream_t stream)
{
    const size_t n = (size_t)H * ((W + 7) / 8) * D;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    fbs::note_launch();
    if (bf16)
        hwd_to_xblock16_kernel<true><<<blocks, 256, 0, stream>>>(in, H, W, D, (__nv_bfloat16*)out);
    else
        hwd_to_xblock16_kernel<false><<<blocks, 256, 0, stream>>>(in, H, W, D, (__half*)out);
    return cudaGetLastError();
}

namespace {

template <bool BF16, int NPT, int PM>
cudaError_t run_tc(const CUtensorMap& map, const CUtensorMap& gmap, const TcParams& p, const TcSmem& L, int grid,
                   float* agg_out, int32_t* disp_int, float* disp_sub, int* err, cudaStream_t stream)
{
    cudaError_t e = fbs::raise_smem_limit(aggregate_tc_kernel<BF16, NPT, PM>, (int)L.total);
    if (e != cudaSuccess) return e;
    // programmatic stream serialization: the kernel may start while the
    // previous kernel of the stream (the cost build, which signals early) ends
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = L.total;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    fbs::note_launch();
    e = cudaLaunchKernelEx(&cfg, aggregate_tc_kernel<BF16, NPT, PM>, map, gmap, p, agg_out, disp_int, disp_sub, err);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// Derived launch parameters; returns false if the case does not fit.
bool tc_plan(int H, int W, int C, int D, int radius, float sigma_s, float sigma_r, bool bf16, TcParams& p,
             TcSmem& L, int max_rows = kMaxR)
{
    if (D < 1 || D > 256 || radius < 0 || radius > 24) return false;
    p.H = H;
    p.W = W;
    p.C = C;
    p.D = D;
    p.N = round_up(D, 16);
    p.Nb = tc_block_rows(D);
    p.split = p.Nb > 256 ? 1 : 0;
    p.rho = radius;
    p.rho8 = round_up(radius, 8);
    p.KW = round_up(16 + p.rho8 + radius, 16);
    p.NH = kTH + 2 * radius;
    p.ntx = (W + kTW - 1) / kTW;
    p.ntiles = p.ntx * ((H + kTH - 1) / kTH);
    const double log2e = 1.4426950408889634;
    p.neg_ks = (float)(-log2e / ((double)sigma_s * sigma_s));
    p.neg_kr = (float)(-log2e / ((double)sigma_r * sigma_r));
    const uint32_t total_n = (uint32_t)p.N + 16;   // disparities + normaliser column block
    p.den_col = (uint32_t)p.N;
    p.nacc = 2 * total_n <= 512 ? 2 : 1;
    p.acc_stride = total_n;
    uint32_t cols = 32;
    while (cols < p.nacc * total_n) cols <<= 1;
    p.tmem_cols = cols;
    p.idesc = tc_idesc(bf16, p.split ? 128 : p.Nb);
    p.idesc2 = tc_idesc(bf16, p.split ? p.Nb - 128 : 16);
    // R window rows per stage and S stages: the largest R (<= kMaxR) with at least
    // 2 stages in 227 KB, then as many stages (<= 6) as fit.  Fewer, larger
    // stages per tile measured faster than deeper pipelines of small stages:
    // each stage costs the producers a wait, a proxy fence and an arrival
    for (p.R = max_rows < 1 || max_rows > kMaxR ? kMaxR : max_rows; p.R >= 1; --p.R) {
        for (p.S = 6; p.S >= 2; --p.S) {
            L = tc_smem_layout(p.KW, p.Nb, p.NH, p.R, p.S);
            if (L.total <= 227 * 1024) return true;
        }
    }
    return false;
}

}  // namespace

int tc_supported(int D, int radius)
{
    TcParams p;
    TcSmem L;
    // resolving the tensor-map encoder here keeps later launches free of
    // driver queries (they may run inside a stream capture)
    return encode_fn() && tc_plan(64, 64, 3, D, radius, 1.f, 1.f, true, p, L) ? 1 : 0;
}

cudaError_t launch_xblock16_pad_rows(int H, int W, int D, bool bf16, void* out, cudaStream_t stream)
{
    const int extra = tc_block_rows(D) - D;
    if (extra <= 0) return cudaSuccess;
    const size_t n = (size_t)H * ((W + 7) / 8) * extra;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    fbs::note_launch();
    if (bf16)
        xblock16_pad_kernel<true><<<blocks, 256, 0, stream>>>(H, W, D, (__nv_bfloat16*)out);
    else
        xblock16_pad_kernel<false><<<blocks, 256, 0, stream>>>(H, W, D, (__half*)out);
    return cudaGetLastError();
}

cudaError_t launch_aggregate_tc(const void* cost, const uint2* rgbx, int H, int W, int C, int D,
                                int radius, float sigma_s, float sigma_r, bool bf16, float* agg_out,
                                int32_t* disp_int, float* disp_sub, int* err, int num_sms, cudaStream_t stream,
                                int max_rows, long long wait_cycles)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    TcParams p;
    TcSmem L;
    if (!tc_plan(H, W, C, D, radius, sigma_s, sigma_r, bf16, p, L, max_rows)) return cudaErrorInvalidValue;
    p.wait_cycles = wait_cycles > 0 ? wait_cycles : kWaitCycles;

    // The two tensor maps depend only on the buffers and the shape: a few
    // recent encodings are kept per host thread (a repeated call with the same
    // buffers, as in a video loop or a benchmark, skips the driver calls).
    struct MapKey {
        const void* cost;
        const void* rgbx;
        int H, W, Nb, KW, NH, R, bf16;
        bool operator==(const MapKey& o) const
        {
            return cost == o.cost && rgbx == o.rgbx && H == o.H && W == o.W && Nb == o.Nb && KW == o.KW &&
                   NH == o.NH && R == o.R && bf16 == o.bf16;
        }
    };
    struct MapEntry {
        MapKey key;
        CUtensorMap map, gmap;
        bool used;
    };
    constexpr int kMapCache = 4;
    thread_local MapEntry cache[kMapCache] = {};
    thread_local int next_slot = 0;
    const MapKey key{cost, rgbx, H, W, p.Nb, p.KW, p.NH, p.R, bf16 ? 1 : 0};
    MapEntry* hit = nullptr;
    for (MapEntry& c : cache)
        if (c.used && c.key == key) hit = &c;
    if (!hit) {
        MapEntry fresh{};
        if (encode_cost_map(enc, &fresh.map, cost, H, W, p.Nb, p.KW, p.R, bf16) != CUDA_SUCCESS ||
            encode_guide_map(enc, &fresh.gmap, rgbx, H, W, rgbx_pitch(W), p.KW, p.NH) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
        fresh.key = key;
        fresh.used = true;
        hit = &cache[next_slot];
        *hit = fresh;
        next_slot = (next_slot + 1) % kMapCache;
    }
    const CUtensorMap& map = hit->map;
    const CUtensorMap& gmap = hit->gmap;

    const int grid = p.ntiles < num_sms ? p.ntiles : num_sms;
    // pairs of window columns per pixel and thread: ceil((radius + 1) / 2).
    // Up to 8 the count is instantiated exactly (an odd radius uses every
    // pair, an even one all but the last pair of phase 1); above, it is
    // rounded up and the surplus pairs are switched off per pair.
    const int npt = (radius + 2) / 2;
    const int pm = (radius & 1) ? 0 : 1;
#define FBS_TC_CASE(n)                                                                                         \
    if (npt == n)                                                                                             \
        return pm == 0 ? (bf16 ? run_tc<true, n, 0>(map, gmap, p, L, grid, agg_out, disp_int, disp_sub, err, stream)  \
                               : run_tc<false, n, 0>(map, gmap, p, L, grid, agg_out, disp_int, disp_sub, err, stream)) \
                       : (bf16 ? run_tc<true, n, 1>(map, gmap, p, L, grid, agg_out, disp_int, disp_sub, err, stream)  \
                               : run_tc<false, n, 1>(map, gmap, p, L, grid, agg_out, disp_int, disp_sub, err, stream));
    FBS_TC_CASE(1)
    FBS_TC_CASE(2)
    FBS_TC_CASE(3)
    FBS_TC_CASE(4)
    FBS_TC_CASE(5)
    FBS_TC_CASE(6)
    FBS_TC_CASE(7)
    FBS_TC_CASE(8)
#undef FBS_TC_CASE
#define FBS_TC_CASE(n)                                                                                     \
    if (npt <= n)                                                                                         \
        return bf16 ? run_tc<true, n, 2>(map, gmap, p, L, grid, agg_out, disp_int, disp_sub, err, stream) \
                    : run_tc<false, n, 2>(map, gmap, p, L, grid, agg_out, disp_int, disp_sub, err, stream);
    FBS_TC_CASE(10)
    FBS_TC_CASE(13)
#undef FBS_TC_CASE
    return cudaErrorInvalidValue;
}

}  // namespace fbs
