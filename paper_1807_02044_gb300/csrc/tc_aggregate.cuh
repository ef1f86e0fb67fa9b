// Pieces shared by the tensor-core aggregation kernels (one pair per launch,
// and the persistent launch over a batch of pairs): the warp roles and tile
// shape, the TMA copies, the bounded waits, the bilateral weights of a column
// pair (Eq. (7)-(8)) and the epilogue's normalisation, WTA and Eq. (10).
// Both kernels call these same functions, so a pixel gets the same bits from
// either of them.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "packed_f32.cuh"
#include "tc_ptx.cuh"

namespace fbs {
namespace tca {

using namespace tc;

constexpr int kTW = 16;         // tile width
constexpr int kTH = 8;          // tile height
constexpr int kM = kTW * kTH;   // 128 = MMA M = TMEM lanes
constexpr int kProducerWarps = 16;                 // warps 0-15
static_assert(kProducerWarps == 16 && kTH == 8 && kTW == 16,
              "producer warp w covers pixel rows 2 (w >> 2), +1 and the stage rows r % 4 == w % 4");
constexpr int kEpiWarp0 = kProducerWarps;          // 4 epilogue warps: TMEM lane quarters 0-3
constexpr int kEpilogue = 128;
constexpr int kTmaWarp = kEpiWarp0 + 4;
constexpr int kMmaWarp = kTmaWarp + 1;
constexpr int kThreads = 32 * (kMmaWarp + 1);
constexpr int kMaxR = 8;          // window rows per stage, at most
// Byte distance between the A operand's core matrices adjacent along K: the
// 2048 bytes of 128 rows x 16 bytes, plus 64 bytes of padding, so that the
// producers' 4-byte stores to the same row of two K-blocks fall in different
// shared-memory banks.
constexpr uint32_t kALbo = 2048 + 64;
constexpr int kMaxRho2 = 2 * 24 + 1;   // row offsets -rho .. rho of the largest radius
// 2^23 as an FP32 bit pattern: for 0 <= c < 2^23 the pattern kMagic + c is the
// float 2^23 + c exactly, so subtracting 2^23 gives float(c) exactly.
constexpr uint32_t kMagic = 0x4B000000u;

inline int round_up(int v, int a) { return (v + a - 1) / a * a; }

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <bool BF16>
struct Op16;
template <>
struct Op16<true> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ T from(float v) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ float to(T v) { return __bfloat162float(v); }
};
template <>
struct Op16<false> {
    using T = __half;
    static __device__ __forceinline__ T from(float v) { return __float2half_rn(v); }
    static __device__ __forceinline__ float to(T v) { return __half2float(v); }
};

// Bounded wait (limit in SM clock cycles) that also gives up as soon as
// another role has aborted.  The waits that only let the CTA's own copies and
// MMAs land before it frees its tensor memory use mbar_wait's fixed ~2 s bound.
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t bar, uint32_t parity, volatile uint32_t* abort_flag,
                                                   long long limit)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (unsigned i = 0; i < kWaitIters; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > limit) break;
    }
    return false;
}
__device__ __forceinline__ void raise_abort(volatile uint32_t* abort_flag, int* err, int code)
{
    if (*abort_flag == 0) *abort_flag = (uint32_t)code;
    atomicCAS(err, 0, code);
}

// The two 16-bit weights of one column pair of one pixel, Eq. (7)-(8).
// Colour distance: |q - p|^2 = |q|^2 + |p|^2 - 2 q.p, exact in integers (|q|^2
// comes with the guide entry, q.p is one dp4a).  It is below 2^23, so carrying
// kMagic in pp = |p|^2 + kMagic turns the integer into the bits of 2^23 + c and
// one packed subtraction (magic2 = -2^23 twice) gives both columns' c as exact
// floats; the exponent argument c * neg_kr + (sx + sy) is one packed FMA.
template <bool BF16>
__device__ __forceinline__ uint32_t tc_weights(const uint4 q, uint32_t pcol, uint32_t pp, uint64_t sxy,
                                               uint64_t magic2, uint64_t nkr2)
{
    const uint32_t e0 = q.y + pp - 2u * __dp4a(q.x, pcol, 0u);
    const uint32_t e1 = q.w + pp - 2u * __dp4a(q.z, pcol, 0u);
    const uint64_t c = f2_add(u2_pack(e0, e1), magic2);
    float a0, a1;
    f2_unpack(f2_fma(c, nkr2, sxy), a0, a1);
    return pack_16x2<BF16>(ex2_approx(a0), ex2_approx(a1));
}

// Byte offsets of a producer thread's column pairs in a window row of the A
// operand.  Pair j covers the columns k = u + 4 j, k + 1 (u = c0 + 2 h, even)
// of pixel row m0, at (k / 8) kALbo + 16 m0 + 2 (k % 8).  With u = 8 a + b,
// an even j = 2 i gives k / 8 = a + i and k % 8 = b; an odd j gives b + 4
// within the same K-block when b < 4, else b - 4 in the next one.  So pair j
// sits at (j odd ? odd : even) + (j / 2) kALbo: two registers and immediate
// offsets instead of one register per pair.
struct TcPairOffsets {
    uint32_t even, odd;
};
__device__ __forceinline__ TcPairOffsets tc_pair_offsets(int u, int m0)
{
    const uint32_t even = (uint32_t)((u >> 3) * kALbo + m0 * 16 + (u & 7) * 2);
    return TcPairOffsets{even, even + ((u & 7) < 4 ? 8u : kALbo - 8u)};
}

// One window row of a producer thread's column pairs: `which` & 1 computes
// the upper pixel (offsets po), & 2 the lower one (+256 bytes); a pixel that
// is not computed gets zeros.  Pair j reads the guide entries at byte 32 j of
// grow and exists when on[j].
template <bool BF16, int NPT>
__device__ __forceinline__ void tc_row_pairs(uint8_t* arow, const uint8_t* grow, const TcPairOffsets po,
                                             const bool (&on)[NPT], const uint64_t (&sxp)[NPT], uint64_t sy0,
                                             uint64_t sy1, int which, uint32_t pcol0, uint32_t pp0, uint32_t pcol1,
                                             uint32_t pp1, uint64_t magic2, uint64_t nkr2)
{
    // at most 5 pairs at a time: their loads first
#pragma unroll
    for (int j0 = 0; j0 < NPT; j0 += 5) {
        uint4 q[5];
        if (which != 0) {
#pragma unroll
            for (int i = 0; i < 5 && j0 + i < NPT; ++i)
                if (on[j0 + i]) q[i] = *(const uint4*)(grow + 32 * (j0 + i));
        }
#pragma unroll
        for (int i = 0; i < 5 && j0 + i < NPT; ++i) {
            const int j = j0 + i;
            if (!on[j]) continue;
            uint8_t* a = arow + ((j & 1) ? po.odd : po.even) + (j >> 1) * kALbo;
            *(uint32_t*)a = (which & 1) ? tc_weights<BF16>(q[i], pcol0, pp0, f2_add(sxp[j], sy0), magic2, nkr2) : 0u;
            *(uint32_t*)(a + 256) =
                (which & 2) ? tc_weights<BF16>(q[i], pcol1, pp1, f2_add(sxp[j], sy1), magic2, nkr2) : 0u;
        }
    }
}

// Normalised aggregated costs of one pixel (the TMEM lane of the calling
// thread) from its accumulator row at tbase: the normaliser in column
// den_col, the N disparity columns from 0.  Writes the D values to arow when
// it is not null, and returns the WTA winner (smallest d on ties) with its
// two neighbours for Eq. (10).
struct TcWta {
    int bidx;
    float best, a_prev, a_next;
};
__device__ __forceinline__ TcWta tc_wta(uint32_t tbase, uint32_t den_col, int N, int D, float* arow)
{
    float dv[16];
    tmem_ld16(tbase + den_col, dv);
    const float inv = 1.f / dv[0];
    const float finf = __int_as_float(0x7f800000);
    float best = finf, a_prev = 0.f, a_next = 0.f, last = 0.f;
    int bidx = 0;
    bool pend = false;   // the best is the previous chunk's last value: its successor comes next
    const uint64_t inv2 = f2_pack(inv, inv);
    // WTA over chunks of 16 values, keeping the neighbours of the running
    // best; two chunks per accumulator read
    for (int c0 = 0; c0 < N; c0 += 32) {
        float v[2][16];
        if (c0 + 16 < N)
            tmem_ld16x2(tbase + (uint32_t)c0, tbase + (uint32_t)c0 + 16, v);
        else
            tmem_ld16(tbase + (uint32_t)c0, v[0]);
#pragma unroll
        for (int hc = 0; hc < 2; ++hc) {
            const int cb = c0 + 16 * hc;
            if (cb >= N) break;
            float* w = v[hc];
#pragma unroll
            for (int i = 0; i < 16; i += 2) f2_unpack(f2_mul(f2_pack(w[i], w[i + 1]), inv2), w[i], w[i + 1]);
            if (arow) {
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (cb + i < D) arow[cb + i] = w[i];
            }
            if (cb + 16 > D) {
                // disparities past D (zero cost rows) never win
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (cb + i >= D) w[i] = finf;
            }
            a_next = pend ? w[0] : a_next;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const bool lt = w[i] < best;
                best = lt ? w[i] : best;
                bidx = lt ? cb + i : bidx;
                a_prev = lt ? (i > 0 ? w[i - 1] : last) : a_prev;
                if (i < 15)
                    a_next = lt ? w[i + 1] : a_next;
                else
                    pend = lt;
            }
            last = w[15];
        }
    }
    return TcWta{bidx, best, a_prev, a_next};
}

// Eq. (10): the vertex of the parabola through the winner and its
// neighbours; the integer winner at the ends of the range or where the
// parabola does not open upwards.
__device__ __forceinline__ float tc_subpixel(const TcWta& r, int D)
{
    float ds = (float)r.bidx;
    if (r.bidx > 0 && r.bidx < D - 1) {
        const float dd = 2.f * r.a_prev + 2.f * r.a_next - 4.f * r.best;
        if (dd > 0.f) ds = (float)r.bidx + (r.a_prev - r.a_next) / dd;
    }
    return ds;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against libcuda); null when the driver does not provide it.
inline EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)f;
    }
    return fn;
}

// The x-blocked 16-bit cost volume as a 4-D tensor: (16 block rows d x 8
// columns = 256 contiguous bytes, group of 16 block rows, block, image row); a
// box covers all Nb block rows of the KW/8 blocks of R window rows and lands
// in shared memory as [R][KW/8][Nb][8], the B operand's K-major core-matrix
// order.  The 256-byte inner dimension keeps the copy at a few wide requests
// per block instead of one per 16-byte block row.
inline CUresult encode_cost_map(EncodeTiledFn enc, CUtensorMap* map, const void* cost, int H, int W, int Nb, int KW,
                                int R, bool bf16)
{
    const int nxb = (W + 7) / 8;
    cuuint64_t dims[4] = {128, (cuuint64_t)(Nb / 16), (cuuint64_t)nxb, (cuuint64_t)H};
    cuuint64_t strides[3] = {256, (cuuint64_t)Nb * 16, (cuuint64_t)nxb * Nb * 16};
    cuuint32_t box[4] = {128, (cuuint32_t)(Nb / 16), (cuuint32_t)(KW / 8), (cuuint32_t)R};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4,
               const_cast<void*>(cost), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

// The packed guide (one 8-byte entry per pixel, row pitch rgbx_pitch(W)) as a
// 2-D tensor; a box is the KW x NH window of a tile.
inline CUresult encode_guide_map(EncodeTiledFn enc, CUtensorMap* map, const uint2* rgbx, int H, int W, int pitch,
                                 int KW, int NH)
{
    cuuint64_t gdims[2] = {(cuuint64_t)W, (cuuint64_t)H};
    cuuint64_t gstrides[1] = {(cuuint64_t)pitch * 8};
    cuuint32_t gbox[2] = {(cuuint32_t)KW, (cuuint32_t)NH};
    cuuint32_t gestr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<uint2*>(rgbx), gdims, gstrides, gbox, gestr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16 (1) or F16 (0),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24
inline uint32_t tc_idesc(bool bf16, int n)
{
    const uint32_t fmt = bf16 ? 1u : 0u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kM >> 4) << 24) | ((uint32_t)(n >> 3) << 17);
}

}  // namespace tca
}  // namespace fbs
