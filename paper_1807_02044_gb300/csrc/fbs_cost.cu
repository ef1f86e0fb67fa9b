// Step 1 of fast bilateral stereo: the matching-cost volume.
//
// NCC (Sec. II-A, Eq. (1)-(3), varrho = 1): with the intensity g taken as the
// channel sum, n = 9 and the block sums S = sum g, Q = sum g^2 and
// P = sum g_l g_r, Eq. (1) multiplied through by n^2 reads
//     c = (n P - S_l S_r) / sqrt((n Q_l - S_l^2) (n Q_r - S_r^2)).
// Every sum and both numerator terms are exact in int32 (g <= 765), so only the
// final normalisation is rounded.  Stored cost: C = 1 - c.  Boundary rules:
// blocks clamp to the image; u - d < 0 gives the maximum cost 2; a block of
// zero variance gives c = 0.
//
// As in the paper (Sec. II-A, Sec. III) the per-pixel block statistics are
// computed once per pixel, so the per-(p, d) work is the dot product P.  Two
// kernels write the two layouts:
//   * cost_kernel, [H][W][ld] float32 (D innermost; the FP32 aggregation),
//     padding d in [D, ld) written as 0.  A pre-pass (grey_stats_kernel: g, S,
//     1/sqrt(nQ - S^2)) fills statistics planes; a thread owns a run of 4
//     pixels and 8 consecutive disparities (left 3x6 grey window in
//     registers, right window sliding one column per disparity, three column
//     products per output column summed by a sliding 3-column window);
//     results are staged in shared memory as [d][x] and written out with D
//     innermost.
//   * cost_xb_kernel, 16-bit x-blocked [H][ceil(W/8)][Dp][8] (the tensor-core
//     aggregation): for a row y and a block of 8 columns, the Dp x 8 block is
//     contiguous, so the tensor-core kernel's TMA reads contiguous blocks that
//     land as K-major core matrices; columns x >= W of the last block are 0.
//     One launch computes the statistics of the rows it stages (a CTA covers
//     up to 4 output rows and stages their grey rows once), the costs (8
//     pixels x 8 disparities per thread), the pad rows D .. Dp-1 and the left
//     image's packed guide.
// Both round the normalisation the same way (ncc_cost), so the 16-bit volume
// equals the FP32 volume rounded to 16 bits.
//
// TAD (not in the paper): C = min(mean_c |I_l(u,v) - I_r(u-d,v)|, tau), tau
// when u - d < 0.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "fbs_internal.cuh"
#include "packed_f32.cuh"

namespace fbs {
namespace {

constexpr int kXS = 128;          // pixels per CTA along x
constexpr int kDC = 64;           // disparities per pass
constexpr int kThreads = 256;     // 32 runs of 4 pixels x 8 groups of 8 disparities
constexpr int kStage = kXS + 1;   // staged row pitch (odd: conflict-free transposed reads)
constexpr int kNRG = kXS + kDC + 2;        // right grey columns per pass
constexpr int kQR = (kNRG + 3) / 4;        // de-interleaved quarter length of a right row
constexpr int kQS = (kXS + kDC) / 4;       // same for the right block statistics

// Lanes of a warp own pixel runs 4*run .. 4*run+3 and read or write column
// 4*run + k together; storing column c at (c & 3) * quarter + (c >> 2) puts
// those 32 accesses in 32 different banks.
__device__ __forceinline__ int stage_pos(int x) { return (x & 3) * 32 + (x >> 2); }
__device__ __forceinline__ int rpos(int c) { return (c & 3) * kQR + (c >> 2); }
__device__ __forceinline__ int spos(int c) { return (c & 3) * kQS + (c >> 2); }

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// C = 1 - c with c = num * (rv_l * rv_r): one rounded product of the two
// normalisers, then one fused multiply-add (every cost kernel uses this, so the
// FP32 and the 16-bit volumes hold the same values before the 16-bit rounding).
__device__ __forceinline__ float ncc_cost(int num, float rv_l, float rv_r)
{
    return __fmaf_rn(-__int2float_rn(num), __fmul_rn(rv_l, rv_r), 1.f);
}

// Per-pixel statistics of one image: g = channel sum, S = 3x3 box sum of g
// (clamped), rv = 1/sqrt(9 Q - S^2) or 0 for a flat block.
__device__ __forceinline__ void stats_pixel(const uint8_t* __restrict__ src, int img, int H, int W, int C, int x,
                                            int y, int16_t* __restrict__ g_out, int* __restrict__ s_out,
                                            float* __restrict__ rv_out, uint2* __restrict__ rgbx)
{
    const size_t plane = (size_t)H * W;
    int s = 0, q = 0;
#pragma unroll
    for (int j = -1; j <= 1; ++j) {
        const int yy = clampi(y + j, 0, H - 1);
#pragma unroll
        for (int k = -1; k <= 1; ++k) {
            const uint8_t* p = src + ((size_t)yy * W + clampi(x + k, 0, W - 1)) * C;
            int g = p[0];
            if (C == 3) g += p[1] + p[2];
            s += g;
            q += g * g;
        }
    }
    const uint8_t* p = src + ((size_t)y * W + x) * C;
    int g = p[0];
    if (C == 3) g += p[1] + p[2];
    if (rgbx != nullptr && img == 0) {
        const uint32_t c = C == 3 ? (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) : (uint32_t)p[0];
        rgbx[(size_t)y * rgbx_pitch(W) + x] = make_uint2(c, (uint32_t)__dp4a(c, c, 0u));
    }
    const int v = 9 * q - s * s;
    const size_t o = img * plane + (size_t)y * W + x;
    g_out[o] = (int16_t)g;
    s_out[o] = s;
    rv_out[o] = v > 0 ? rsqrtf((float)v) : 0.f;
}

__global__ void __launch_bounds__(256)
grey_stats_kernel(const uint8_t* __restrict__ L, const uint8_t* __restrict__ R, int H, int W, int C,
                  int16_t* __restrict__ g_out, int* __restrict__ s_out, float* __restrict__ rv_out,
                  uint2* __restrict__ rgbx)
{
    const int img = blockIdx.z;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= W) return;
    stats_pixel(img == 0 ? L : R, img, H, W, C, x, blockIdx.y, g_out, s_out, rv_out, rgbx);
}

// Batched statistics: an item is one row of one pair (both images).
__global__ void __launch_bounds__(256)
grey_stats_batched_kernel(const BatchPair* __restrict__ pairs, int npairs, int nitems, int* __restrict__ counter)
{
    __shared__ int item_s;
    for (;;) {
        if (threadIdx.x == 0) item_s = atomicAdd(counter, 1);
        __syncthreads();
        const int item = item_s;
        __syncthreads();
        if (item >= nitems) break;
        const BatchPair& bp = pairs[find_pair(pairs, npairs, item, &BatchPair::stat_off)];
        const int y = item - bp.stat_off;
        if (bp.mode != 0) continue;   // TAD needs no statistics
        for (int x = threadIdx.x; x < bp.W; x += blockDim.x)
            for (int img = 0; img < 2; ++img)
                stats_pixel(img == 0 ? bp.left : bp.right, img, bp.H, bp.W, bp.C, x, y, bp.sc.g, bp.sc.s, bp.sc.rv,
                            bp.sc.rgbx);
    }
}

template <typename T>
__device__ __forceinline__ T to_out(float v);
template <>
__device__ __forceinline__ float to_out<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_out<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half to_out<__half>(float v) { return __float2half_rn(v); }

template <typename T>
__device__ __forceinline__ uint4 pack8(const T (&v)[8])
{
    static_assert(sizeof(T) == 2, "16-bit values");
    uint32_t w[4];
#pragma unroll
    for (int c = 0; c < 4; ++c)
        w[c] = (uint32_t)*reinterpret_cast<const unsigned short*>(&v[2 * c]) |
               ((uint32_t)*reinterpret_cast<const unsigned short*>(&v[2 * c + 1]) << 16);
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// MODE 0: NCC from the statistics planes; MODE 1: TAD from the raw images.
// out is [H][W][ld] (T = float).
// One row y and 128 pixels from x0, disparities [d_begin, d_end) (all: 0, D);
// ends with a __syncthreads.  out_r (nullable, FP32 layout only): the right
// view's volume, which holds the same costs at (x - d, y, d) (Sec. II-A, Sec. III).
template <int MODE, typename T>
__device__ __forceinline__ void cost_tile(const int16_t* __restrict__ gplane, const int* __restrict__ splane,
                                          const float* __restrict__ rvplane, const uint8_t* __restrict__ L,
                                          const uint8_t* __restrict__ R, int H, int W, int C, int D, int ld, float tau,
                                          T* __restrict__ out, int x0, int y, int* smem_i, int d_begin, int d_end,
                                          float* __restrict__ out_r = nullptr)
{
    const int tid = threadIdx.x;
    const int nxs = min(kXS, W - x0);
    const size_t plane = (size_t)H * W;
    // layout: stage [kDC][kStage] float | left grey [3][kXS+2] | right grey [3][kXS+kDC+2] |
    //         S_l, rv_l [kXS] | S_r, rv_r [kXS+kDC]
    float* stage = (float*)smem_i;
    int* gl = (int*)(stage + kDC * kStage);
    int* gr = gl + 3 * (kXS + 2);      // [3][4 * kQR], column c at rpos(c)
    int* sl = gr + 3 * 4 * kQR;
    float* rl = (float*)(sl + kXS);
    int* sr = (int*)(rl + kXS);
    float* rr = (float*)(sr + kXS + kDC);
    uchar4* pl = (uchar4*)gl;          // TAD: raw left row [kXS]
    uchar4* pr = pl + kXS;             // TAD: raw right row [kXS + kDC]

    const int run = tid & 31;          // pixels 4*run .. 4*run+3 of the CTA
    const int dg = tid >> 5;           // disparities dc + 8*dg .. +7
    const int xl0 = 4 * run;

    if (MODE == 0) {
        // left grey window rows y-1..y+1, virtual columns x0-1 .. x0+kXS
        for (int i = tid; i < 3 * (kXS + 2); i += kThreads) {
            const int j = i / (kXS + 2), c = i - j * (kXS + 2);
            gl[i] = gplane[(size_t)clampi(y - 1 + j, 0, H - 1) * W + clampi(x0 - 1 + c, 0, W - 1)];
        }
        for (int i = tid; i < kXS; i += kThreads) {
            const int x = clampi(x0 + i, 0, W - 1);
            sl[i] = splane[(size_t)y * W + x];
            rl[i] = rvplane[(size_t)y * W + x];
        }
    } else {
        for (int i = tid; i < kXS; i += kThreads) {
            const uint8_t* p = L + ((size_t)y * W + clampi(x0 + i, 0, W - 1)) * C;
            pl[i] = C == 3 ? make_uchar4(p[0], p[1], p[2], 0) : make_uchar4(p[0], 0, 0, 0);
        }
    }

    for (int dc = d_begin; dc < d_end; dc += kDC) {
        // right columns for this pass: virtual columns rb .. rb + NRG - 1 with
        // rb = x0 - dc - kDC - 1; the right block of (x, d) spans x-d-1 .. x-d+1
        const int rb = x0 - dc - kDC - 1;
        if (MODE == 0) {
            for (int i = tid; i < 3 * kNRG; i += kThreads) {
                const int j = i / kNRG, c = i - j * kNRG;
                gr[j * 4 * kQR + rpos(c)] =
                    gplane[plane + (size_t)clampi(y - 1 + j, 0, H - 1) * W + clampi(rb + c, 0, W - 1)];
            }
            // right block centres rb+1 .. rb+kXS+kDC
            for (int i = tid; i < kXS + kDC; i += kThreads) {
                const int x = clampi(rb + 1 + i, 0, W - 1);
                sr[spos(i)] = splane[plane + (size_t)y * W + x];
                rr[spos(i)] = rvplane[plane + (size_t)y * W + x];
            }
        } else {
            for (int i = tid; i < kXS + kDC; i += kThreads) {
                const uint8_t* p = R + ((size_t)y * W + clampi(rb + 1 + i, 0, W - 1)) * C;
                pr[i] = C == 3 ? make_uchar4(p[0], p[1], p[2], 0) : make_uchar4(p[0], 0, 0, 0);
            }
        }
        __syncthreads();

        const int d_first = dc + 8 * dg;
        if (MODE == 0) {
            int glw[3][6];
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int c = 0; c < 6; ++c) glw[j][c] = gl[j * (kXS + 2) + xl0 + c];
            int sli[4];
            float rli[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                sli[i] = sl[xl0 + i];
                rli[i] = rl[xl0 + i];
            }
            // right window for d_first: virtual columns x0+xl0-d-1 .. +4, index (col - rb)
            int grw[3][6];
            int srw[4];
            float rrw[4];
            {
                const int base = x0 + xl0 - d_first - 1 - rb;
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int c = 0; c < 6; ++c) grw[j][c] = gr[j * 4 * kQR + rpos(base + c)];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    srw[i] = sr[spos(base + i)];
                    rrw[i] = rr[spos(base + i)];
                }
            }
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                const int d = d_first + s;
                if (s > 0) {
                    // slide one column to the left: d grew by one
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
#pragma unroll
                        for (int c = 5; c > 0; --c) grw[j][c] = grw[j][c - 1];
                    }
                    const int base = x0 + xl0 - d - 1 - rb;
#pragma unroll
                    for (int j = 0; j < 3; ++j) grw[j][0] = gr[j * 4 * kQR + rpos(base)];
#pragma unroll
                    for (int i = 3; i > 0; --i) {
                        srw[i] = srw[i - 1];
                        rrw[i] = rrw[i - 1];
                    }
                    srw[0] = sr[spos(base)];
                    rrw[0] = rr[spos(base)];
                }
                int cp[6];
#pragma unroll
                for (int c = 0; c < 6; ++c) cp[c] = glw[0][c] * grw[0][c] + glw[1][c] * grw[1][c] + glw[2][c] * grw[2][c];
                float* st = stage + (d - dc) * kStage + run;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int x = x0 + xl0 + i;
                    const int num = 9 * (cp[i] + cp[i + 1] + cp[i + 2]) - sli[i] * srw[i];
                    st[32 * i] = x - d < 0 ? 2.f : ncc_cost(num, rli[i], rrw[i]);
                }
            }
        } else {
            const float inv_c = 1.f / (float)C;
#pragma unroll 2
            for (int s = 0; s < 8; ++s) {
                const int d = d_first + s;
                float* st = stage + (d - dc) * kStage + run;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int x = x0 + xl0 + i;
                    float cst = tau;
                    if (x - d >= 0) {
                        const uchar4 a = pl[xl0 + i];
                        const uchar4 b = pr[x - d - (rb + 1)];
                        const int sad = abs((int)a.x - (int)b.x) + abs((int)a.y - (int)b.y) + abs((int)a.z - (int)b.z);
                        cst = fminf((float)sad * inv_c, tau);
                    }
                    st[32 * i] = cst;
                }
            }
        }
        __syncthreads();

        const int nd = min(kDC, d_end - dc);
        // out[(y*W + x)*ld + d]; padding d in [D, ld) of the last pass written as 0
        const int ndw = (dc + kDC >= d_end) ? (d_end == D ? ld - dc : d_end - dc) : kDC;
        const int warp = tid >> 5, lane = tid & 31;
        for (int x = warp; x < nxs; x += kThreads / 32) {
            T* o = out + ((size_t)y * W + x0 + x) * ld + dc;
            const int px = stage_pos(x);
            for (int dd = lane; dd < ndw; dd += 32) o[dd] = to_out<T>(dd < nd ? stage[dd * kStage + px] : 0.f);
        }
        if (out_r != nullptr) {
            // right pixel xr = x - d receives the contiguous disparities
            // max(dc, x0 - xr) .. min(dc + nd - 1, x0 + nxs - 1 - xr) of this pass
            const int xr_lo = max(0, x0 - dc - nd + 1), xr_hi = x0 + nxs - 1 - dc;
            for (int xr = xr_lo + warp; xr <= xr_hi; xr += kThreads / 32) {
                const int dlo = max(dc, x0 - xr), dhi = min(dc + nd - 1, x0 + nxs - 1 - xr);
                float* o = out_r + ((size_t)y * W + xr) * ld;
                for (int d = dlo + lane; d <= dhi; d += 32) o[d] = stage[(d - dc) * kStage + stage_pos(xr + d - x0)];
            }
        }
        __syncthreads();
    }
}

template <int MODE, typename T>
__global__ void __launch_bounds__(kThreads)
cost_kernel(const int16_t* __restrict__ gplane, const int* __restrict__ splane, const float* __restrict__ rvplane,
            const uint8_t* __restrict__ L, const uint8_t* __restrict__ R, int H, int W, int C, int D, int ld,
            float tau, T* __restrict__ out)
{
    extern __shared__ int smem_i[];
    cost_tile<MODE, T>(gplane, splane, rvplane, L, R, H, W, C, D, ld, tau, out, blockIdx.x * kXS, blockIdx.y,
                               smem_i, 0, D);
}

// Batched FP32 cost volumes [H][W][ld]: an item is (row, 128-pixel segment) of a pair.
__global__ void __launch_bounds__(kThreads)
cost_batched_kernel(const BatchPair* __restrict__ pairs, int npairs, int nitems, int* __restrict__ counter)
{
    extern __shared__ int smem_i[];
    __shared__ int item_s;
    for (;;) {
        if (threadIdx.x == 0) item_s = atomicAdd(counter, 1);
        __syncthreads();
        const int item = item_s;
        __syncthreads();
        if (item >= nitems) break;
        const BatchPair& bp = pairs[find_pair(pairs, npairs, item, &BatchPair::cost_off)];
        const int t = item - bp.cost_off;
        const int nseg = (bp.W + kXS - 1) / kXS;
        const int x0 = (t % nseg) * kXS, y = t / nseg;
        if (bp.mode == 0)
            cost_tile<0, float>(bp.sc.g, bp.sc.s, bp.sc.rv, bp.left, bp.right, bp.H, bp.W, bp.C, bp.D, bp.ld,
                                       bp.tau, bp.cost, x0, y, smem_i, 0, bp.D);
        else
            cost_tile<1, float>(bp.sc.g, bp.sc.s, bp.sc.rv, bp.left, bp.right, bp.H, bp.W, bp.C, bp.D, bp.ld,
                                       bp.tau, bp.cost, x0, y, smem_i, 0, bp.D);
    }
}

// Band form: NCC costs of row y, pixels x0 .. x0+127, for the disparities
// that some aggregation tile reading this segment needs: the hull of the
// ranges [d_begin, d_end) of every tile whose window halo (the tile grown by
// rho) overlaps the segment.  Entries outside that hull are not written.
__global__ void __launch_bounds__(kThreads)
cost_band_kernel(const int16_t* __restrict__ gplane, const int* __restrict__ splane,
                 const float* __restrict__ rvplane, int H, int W, int D, int ld, int rho,
                 const int2* __restrict__ tile_range, int ntx, int nty, float* __restrict__ out)
{
    extern __shared__ int smem_i[];
    __shared__ int lo_s, hi_s;
    const int x0 = blockIdx.x * kXS, y = blockIdx.y;
    if (threadIdx.x == 0) {
        lo_s = D;
        hi_s = 0;
    }
    __syncthreads();
    // tiles ty with 4ty - rho <= y <= 4ty + 3 + rho, tx with halo columns meeting [x0, x0 + 127]
    const int ty0 = max(0, (y - rho + kAggTileY * 64) / kAggTileY - 64);
    const int ty1 = min(nty - 1, (y + rho) / kAggTileY);
    const int tx0 = max(0, (x0 - rho + kAggTileX * 64) / kAggTileX - 64);
    const int tx1 = min(ntx - 1, (x0 + kXS - 1 + rho) / kAggTileX);
    const int nx = tx1 - tx0 + 1;
    int lo = D, hi = 0;
    for (int i = threadIdx.x; i < (ty1 - ty0 + 1) * nx; i += kThreads) {
        const int2 r = tile_range[(size_t)(ty0 + i / nx) * ntx + tx0 + i % nx];
        lo = min(lo, r.x);
        hi = max(hi, r.y);
    }
    if (ty0 <= ty1 && tx0 <= tx1) {
        atomicMin(&lo_s, lo);
        atomicMax(&hi_s, hi);
    }
    __syncthreads();
    const int d_begin = lo_s, d_end = hi_s;
    if (d_begin >= d_end) return;
    cost_tile<0, float>(gplane, splane, rvplane, nullptr, nullptr, H, W, 1, D, ld, 0.f, out, x0, y, smem_i,
                               d_begin, d_end);
}

// Both views at once (FP32 layouts): the left volume as cost_kernel writes it
// and the right volume from the same staged costs.
template <int MODE>
__global__ void __launch_bounds__(kThreads)
cost_lr_kernel(const int16_t* __restrict__ gplane, const int* __restrict__ splane, const float* __restrict__ rvplane,
               const uint8_t* __restrict__ L, const uint8_t* __restrict__ R, int H, int W, int C, int D, int ld,
               float tau, float* __restrict__ out, float* __restrict__ out_r)
{
    extern __shared__ int smem_i[];
    cost_tile<MODE, float>(gplane, splane, rvplane, L, R, H, W, C, D, ld, tau, out, blockIdx.x * kXS, blockIdx.y,
                                  smem_i, 0, D, out_r);
}

// Right volume entries with no left pixel (xr + d >= W): the maximum cost;
// d in [D, ld) padding: 0.
__global__ void right_edge_fill_kernel(int H, int W, int D, int ld, float maxc, float* __restrict__ out_r)
{
    const int y = blockIdx.x;
    const int x_first = max(0, W - D);
    const int n = (W - x_first) * ld;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int xr = x_first + i / ld, d = i % ld;
        if (d >= D) out_r[((size_t)y * W + xr) * ld + d] = 0.f;
        else if (xr + d >= W) out_r[((size_t)y * W + xr) * ld + d] = maxc;
    }
}

// ---- 16-bit x-blocked volume: one thread per (block of 8 columns, 8 disparities)
//
// The layout [H][ceil(W/8)][Dp][8] keeps the 8 columns of a block contiguous
// for each d, so a thread that owns one block and 8 consecutive disparities
// computes the 8 x 8 costs in registers, one 16-byte row per d.  Lanes own
// consecutive disparity groups of a block; the warp passes its 256 rows
// through a private shared-memory buffer so that each store instruction
// writes 32 consecutive rows (512 contiguous bytes within a block).  The left 3x10 grey window and the left
// statistics stay in registers; the right window (3x10 values and 8 block
// statistics) slides one column per disparity, 5 new shared-memory values.
// Per (p, d): three multiply-adds per column product shared by three pixels,
// the sliding 3-column sum, the numerator and ncc_cost -- about 10
// instructions.  Staged rows use a skewed index c + c/8, so lanes reading
// columns 8 apart hit different banks.
constexpr int kXbThreads = 256;

__device__ __forceinline__ int skew(int c) { return c + (c >> 3); }
__host__ __device__ inline int skew_len(int n) { return n + (n - 1) / 8; }

// x-blocks per CTA: 16 up to 8 disparity groups, then 8 (measured best on
// GB300 for D = 64, 128 and 256; smaller CTAs interleave their staging and
// compute phases better, and 640 columns split evenly into 16-block CTAs)
__host__ __device__ inline int xb_blocks_per_cta(int D)
{
    const int ndg = (D + 7) / 8;
    const int b = ndg <= 8 ? 16 : 8;
    return b * ndg <= kXbThreads ? b : kXbThreads / ndg;
}

// Per-warp output buffer: 256 rows of 16 bytes, row r at r + r/8 (conflict-free
// both when lanes write their 8 rows and when the warp reads 32 consecutive rows).
constexpr int kXbWarpRows = 256 + 32;

// Output rows per CTA (1, 2 or 4, chosen at launch): the CTA stages grey rows
// y0-1 .. y0+rows once for all of them (rows + 2 rows of each image instead of
// 3 per output row).
constexpr int kXbMaxRows = 4;

__host__ __device__ inline size_t cost_xb_stage_ints(int mode, int D, int rows)
{
    const int npx = 8 * xb_blocks_per_cta(D);
    const int Ll = skew_len(npx + 2), Lr = skew_len(npx + D + 9), Lp = skew_len(npx);
    // NCC: grey rows of both images, then per output row the left and right
    // block statistics; TAD: per output row the packed pixels of both images
    const size_t n = mode == 0 ? (size_t)((rows + 2) * (Ll + Lr) + rows * (2 * Lp + 2 * Lr))
                               : (size_t)rows * (Lp + Lr);
    return (n + 3) & ~(size_t)3;   // the output buffers that follow are 16-byte aligned
}

template <int MODE, typename T>
__global__ void __launch_bounds__(kXbThreads, 2)
cost_xb_kernel(const uint8_t* __restrict__ L, const uint8_t* __restrict__ R, int H, int W, int C, int D, float tau,
               T* __restrict__ out, uint2* __restrict__ rgbx, int rows)
{
    extern __shared__ int sm_xb[];
    // let a programmatically launched successor (the tensor-core aggregation)
    // start its set-up once every CTA of this grid has started; it waits for
    // this grid's completion before it reads anything this kernel writes
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int ndg = (D + 7) >> 3;
    const int xbc = xb_blocks_per_cta(D);
    const int nxb = (W + 7) >> 3;
    const int xb0 = blockIdx.x * xbc;
    const int y0 = blockIdx.y * rows;
    const int nrows = min(rows, H - y0);
    const int x0 = xb0 * 8;
    const int npx = xbc * 8;
    const int nl = npx + 2;            // left grey columns x0-1 .. x0+npx
    // right columns x0-D-8 .. x0+npx (origin rb): the 8 extra columns keep every
    // index of a thread's 8 disparities >= 0 also past D (those rows are not stored)
    const int nr = npx + D + 9;
    const int rb = x0 - D - 8;
    const int Ll = skew_len(nl), Lr = skew_len(nr), Lp = skew_len(npx);

    int* gl = sm_xb;                             // [rows + 2][Ll]: grey rows y0-1 ..
    int* gr = gl + (rows + 2) * Ll;              // [rows + 2][Lr]
    int* sl = gr + (rows + 2) * Lr;              // [rows][Lp]
    float* rl = (float*)(sl + rows * Lp);        // [rows][Lp]
    int* sr = (int*)(rl + rows * Lp);            // [rows][Lr]
    float* rr = (float*)(sr + rows * Lr);        // [rows][Lr]
    uint32_t* pl = (uint32_t*)sm_xb;             // TAD: left pixels [rows][Lp]
    uint32_t* pr = pl + rows * Lp;               // TAD: right pixels [rows][Lr], origin rb

    // staging: grey values (channel sums) of rows y0-1 .. y0+nrows at clamped
    // columns, then for each output row the statistics S, 1/sqrt(9Q - S^2) of
    // every staged block centre exactly as grey_stats_kernel computes them, and
    // the left pixels' packed guide
    auto grey = [&](const uint8_t* img, int yy, int x) -> int {
        const uint8_t* q = img + ((size_t)yy * W + x) * C;
        return C == 3 ? (int)q[0] + (int)q[1] + (int)q[2] : (int)q[0];
    };
    auto colour = [&](const uint8_t* img, int yy, int x) -> uint32_t {
        const uint8_t* q = img + ((size_t)yy * W + clampi(x, 0, W - 1)) * C;
        return C == 3 ? (uint32_t)q[0] | ((uint32_t)q[1] << 8) | ((uint32_t)q[2] << 16) : (uint32_t)q[0];
    };
    if (MODE == 0) {
        for (int c = tid; c < nl; c += nthr) {
            const int x = clampi(x0 - 1 + c, 0, W - 1);
            for (int j = 0; j < nrows + 2; ++j) gl[j * Ll + skew(c)] = grey(L, clampi(y0 - 1 + j, 0, H - 1), x);
        }
        for (int c = tid; c < nr; c += nthr) {
            const int x = clampi(rb + c, 0, W - 1);
            for (int j = 0; j < nrows + 2; ++j) gr[j * Lr + skew(c)] = grey(R, clampi(y0 - 1 + j, 0, H - 1), x);
        }
        __syncthreads();
        for (int e = tid; e < nrows * npx; e += nthr) {
            // left centre x0 + i of output row k sits at staged column i + 1 of rows k .. k+2
            const int k = e / npx, i = e - k * npx;
            const int* g = gl + k * Ll;
            int sum = 0, sq = 0;
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const int v = g[j * Ll + skew(i + m)];
                    sum += v;
                    sq += v * v;
                }
            const int var = 9 * sq - sum * sum;
            sl[k * Lp + skew(i)] = sum;
            rl[k * Lp + skew(i)] = var > 0 ? rsqrtf((float)var) : 0.f;
            if (x0 + i < W) {
                const uint32_t col = colour(L, y0 + k, x0 + i);
                rgbx[(size_t)(y0 + k) * rgbx_pitch(W) + x0 + i] = make_uint2(col, (uint32_t)__dp4a(col, col, 0u));
            }
        }
        for (int e = tid; e < nrows * (nr - 2); e += nthr) {
            const int k = e / (nr - 2), c = 1 + e - k * (nr - 2);
            const int* g = gr + k * Lr;
            int sum = 0, sq = 0;
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int m = -1; m <= 1; ++m) {
                    const int v = g[j * Lr + skew(c + m)];
                    sum += v;
                    sq += v * v;
                }
            const int var = 9 * sq - sum * sum;
            sr[k * Lr + skew(c)] = sum;
            rr[k * Lr + skew(c)] = var > 0 ? rsqrtf((float)var) : 0.f;
        }
    } else {
        for (int e = tid; e < nrows * npx; e += nthr) {
            const int k = e / npx, c = e - k * npx;
            const uint32_t col = colour(L, y0 + k, x0 + c);
            pl[k * Lp + skew(c)] = col;
            if (x0 + c < W)
                rgbx[(size_t)(y0 + k) * rgbx_pitch(W) + x0 + c] = make_uint2(col, (uint32_t)__dp4a(col, col, 0u));
        }
        for (int e = tid; e < nrows * nr; e += nthr) {
            const int k = e / nr, c = e - k * nr;
            pr[k * Lr + skew(c)] = colour(R, y0 + k, rb + c);
        }
    }
    __syncthreads();

    const int dg = tid % ndg, xbl = tid / ndg;
    const int xb = xb0 + xbl;
    // threads past xbc * ndg (the block is a whole number of warps) and blocks
    // beyond the image compute nothing and store nothing
    const bool active = xbl < xbc && xb < nxb;
    const int d0 = 8 * dg;
    const int xl = 8 * xbl;            // the block's first pixel, relative to x0
    const int xbase = x0 + xl;
    const int lane = tid & 31;
    constexpr bool kBf16 = std::is_same<T, __nv_bfloat16>::value;
    uint4* wbuf = (uint4*)(sm_xb + cost_xb_stage_ints(MODE, D, rows)) + (size_t)(tid >> 5) * kXbWarpRows;
    uint4* mine = wbuf + 9 * lane;     // rows 8*lane + s at 9*lane + s

    for (int k = 0; k < nrows; ++k) {
        const int y = y0 + k;
        // this output row's staged rows (grey rows k .. k+2 are y-1 .. y+1) and statistics
        const int* glk = gl + k * Ll;
        const int* grk = gr + k * Lr;
        const int* slk = sl + k * Lp;
        const float* rlk = rl + k * Lp;
        const int* srk = sr + k * Lr;
        const float* rrk = rr + k * Lr;
        const uint32_t* plk = pl + k * Lp;
        const uint32_t* prk = pr + k * Lr;
        (void)glk, (void)grk, (void)slk, (void)rlk, (void)srk, (void)rrk, (void)plk, (void)prk;
        if (!active) {
        } else if (MODE == 0) {
            int glw[3][10], grw[3][10], sli[8], srw[8];
            float rli[8], rrw[8];
    #pragma unroll
            for (int j = 0; j < 3; ++j)
    #pragma unroll
                for (int c = 0; c < 10; ++c) glw[j][c] = glk[j * Ll + skew(xl + c)];
    #pragma unroll
            for (int i = 0; i < 8; ++i) {
                sli[i] = slk[skew(xl + i)];
                rli[i] = rlk[skew(xl + i)];
            }
            // right block of (x, d) spans columns x-d-1 .. x-d+1: index (x - d - 1 + k) - rb
            int base = xl - d0 - 1 + D + 8;
    #pragma unroll
            for (int j = 0; j < 3; ++j)
    #pragma unroll
                for (int c = 0; c < 10; ++c) grw[j][c] = grk[j * Lr + skew(base + c)];
    #pragma unroll
            for (int i = 0; i < 8; ++i) {
                srw[i] = srk[skew(base + 1 + i)];
                rrw[i] = rrk[skew(base + 1 + i)];
            }
            // the normalisation of a pixel pair is one packed multiply and one packed
            // FMA (per lane exactly ncc_cost); threads whose 8 pixels are inside the
            // image and match inside it for all 8 disparities skip the two masks
            const uint64_t ones2 = f2_pack(1.f, 1.f);
            auto sweep = [&](auto masked) {
    #pragma unroll
                for (int s = 0; s < 8; ++s) {
                    const int d = d0 + s;
                    if (s > 0) {
                        // d grew by one: the window slides one column to the left
                        --base;
    #pragma unroll
                        for (int j = 0; j < 3; ++j) {
    #pragma unroll
                            for (int c = 9; c > 0; --c) grw[j][c] = grw[j][c - 1];
                            grw[j][0] = grk[j * Lr + skew(base)];
                        }
    #pragma unroll
                        for (int i = 7; i > 0; --i) {
                            srw[i] = srw[i - 1];
                            rrw[i] = rrw[i - 1];
                        }
                        srw[0] = srk[skew(base + 1)];
                        rrw[0] = rrk[skew(base + 1)];
                    }
                    int cp[10];
    #pragma unroll
                    for (int c = 0; c < 10; ++c)
                        cp[c] = glw[0][c] * grw[0][c] + glw[1][c] * grw[1][c] + glw[2][c] * grw[2][c];
                    int P = cp[0] + cp[1] + cp[2];
                    int num[8];
    #pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        if (i > 0) P += cp[i + 2] - cp[i - 1];
                        num[i] = 9 * P - sli[i] * srw[i];
                    }
                    uint32_t w[4];
    #pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const uint64_t t = f2_mul(f2_pack(rli[2 * q], rli[2 * q + 1]), f2_pack(rrw[2 * q], rrw[2 * q + 1]));
                        const uint64_t nn = f2_pack(-__int2float_rn(num[2 * q]), -__int2float_rn(num[2 * q + 1]));
                        float c0, c1;
                        f2_unpack(f2_fma(nn, t, ones2), c0, c1);
                        if (decltype(masked)::value) {
                            const int x = xbase + 2 * q;
                            c0 = x - d < 0 ? 2.f : c0;
                            c1 = x + 1 - d < 0 ? 2.f : c1;
                            c0 = x < W ? c0 : 0.f;
                            c1 = x + 1 < W ? c1 : 0.f;
                        }
                        w[q] = pack_16x2<kBf16>(c0, c1);
                    }
                    mine[s] = make_uint4(w[0], w[1], w[2], w[3]);
                }
            };
            if (xbase + 7 < W && xbase >= d0 + 7)
                sweep(std::integral_constant<bool, false>{});
            else
                sweep(std::integral_constant<bool, true>{});
        } else {
            const float inv_c = 1.f / (float)C;
            uint32_t pli[8], prw[8];
    #pragma unroll
            for (int i = 0; i < 8; ++i) pli[i] = plk[skew(xl + i)];
            // right pixel of (x, d): index (x - d) - rb
            int base = xl - d0 + D + 8;
    #pragma unroll
            for (int i = 0; i < 8; ++i) prw[i] = prk[skew(base + i)];
    #pragma unroll
            for (int s = 0; s < 8; ++s) {
                const int d = d0 + s;
                if (s > 0) {
                    --base;
    #pragma unroll
                    for (int i = 7; i > 0; --i) prw[i] = prw[i - 1];
                    prw[0] = prk[skew(base)];
                }
                T v[8];
    #pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int x = xbase + i;
                    const int sad = (int)__dp4a(__vabsdiffu4(pli[i], prw[i]), 0x01010101u, 0u);
                    const float cst = x - d < 0 ? tau : fminf((float)sad * inv_c, tau);
                    v[i] = to_out<T>(x < W ? cst : 0.f);
                }
                mine[s] = pack8(v);
            }
        }
        // write-out: entry e = 32k + lane is row s = e % 8 of lane e / 8 (its block
        // xbl and group dg come by shuffle); rows d >= D and inactive lanes are skipped
        __syncwarp();
        const int Dp = tc_block_rows(D);
        const int code = active ? (xbl << 8) | dg : -1;
    #pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int e = 32 * k + lane;
            const int src = __shfl_sync(0xffffffffu, code, e >> 3);
            const int s = e & 7;
            if (src >= 0 && 8 * (src & 255) + s < D) {
                const int xbs = xb0 + (src >> 8);
                const uint4 row = wbuf[e + (e >> 3)];
                *(uint4*)(out + (((size_t)y * nxb + xbs) * Dp + 8 * (src & 255) + s) * 8) = row;
            }
        }
        // rows D .. Dp-1 of the CTA's blocks: zero, except row round_up(D,16) all
        // ones when the normaliser rides with the volume
        const int extra = Dp - D;
        if (extra > 0) {
            const int n16 = (D + 15) / 16 * 16;
            const T one1[2] = {to_out<T>(1.f), to_out<T>(1.f)};
            const uint32_t ones = *reinterpret_cast<const uint32_t*>(one1);
            const int nb = min(xbc, nxb - xb0);
            for (int i = tid; i < nb * extra; i += nthr) {
                const int b = i / extra, d = D + (i - b * extra);
                const uint32_t v = (d == n16 && Dp > n16) ? ones : 0u;
                *(uint4*)(out + (((size_t)y * nxb + xb0 + b) * Dp + d) * 8) = make_uint4(v, v, v, v);
            }
        }
        __syncwarp();   // the warp's buffer is read out before the next row's sweep refills it
    }
}

size_t cost_xb_smem_bytes(int mode, int D, int rows)
{
    const int nwarps = (xb_blocks_per_cta(D) * ((D + 7) / 8) + 31) / 32;
    return sizeof(int) * cost_xb_stage_ints(mode, D, rows) + (size_t)nwarps * kXbWarpRows * 16;
}

template <int MODE, typename T>
cudaError_t launch_cost_xb(const CostScratch& sc, const uint8_t* left, const uint8_t* right, int H, int W, int C,
                           int D, float tau, T* out, cudaStream_t stream)
{
    const int ndg = (D + 7) / 8;
    const int xbc = xb_blocks_per_cta(D);
    const int nxb = (W + 7) / 8;
    const int gx = (nxb + xbc - 1) / xbc;
    // the most rows per CTA that still leave about four CTAs per SM (small
    // images need the CTAs more than the shared staging)
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int rows = kXbMaxRows;
    while (rows > 1 && (long long)gx * ((H + rows - 1) / rows) < 4LL * sms) rows /= 2;
    const size_t smem = cost_xb_smem_bytes(MODE, D, rows);
    e = fbs::raise_smem_limit(cost_xb_kernel<MODE, T>, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(gx, (H + rows - 1) / rows);
    fbs::note_launch();
    const int nthr = (xbc * ndg + 31) / 32 * 32;   // whole warps (the write-out shuffles need all lanes)
    cost_xb_kernel<MODE, T><<<grid, nthr, smem, stream>>>(left, right, H, W, C, D, tau, out, sc.rgbx, rows);
    return cudaGetLastError();
}

size_t cost_smem_bytes()
{
    return sizeof(float) * (size_t)kDC * kStage +
           sizeof(int) * (size_t)(3 * (kXS + 2) + 3 * 4 * kQR + 2 * kXS + 2 * (kXS + kDC));
}

template <int MODE, typename T>
cudaError_t launch_cost_kernel(const CostScratch& sc, const uint8_t* left, const uint8_t* right, int H, int W,
                               int C, int D, int ld, float tau, T* out, cudaStream_t stream)
{
    const size_t smem = cost_smem_bytes();
    cudaError_t e = fbs::raise_smem_limit(cost_kernel<MODE, T>, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((W + kXS - 1) / kXS, H);
    fbs::note_launch();
    cost_kernel<MODE, T><<<grid, kThreads, smem, stream>>>(sc.g, sc.s, sc.rv, left, right, H, W, C, D, ld,
                                                                   tau, out);
    return cudaGetLastError();
}

cudaError_t launch_stats(const CostScratch& sc, const uint8_t* left, const uint8_t* right, int H, int W, int C,
                         cudaStream_t stream)
{
    dim3 grid((W + 255) / 256, H, 2);
    fbs::note_launch();
    grey_stats_kernel<<<grid, 256, 0, stream>>>(left, right, H, W, C, sc.g, sc.s, sc.rv, sc.rgbx);
    return cudaGetLastError();
}

}  // namespace

int stats_items(int H, int W) { return H; }
int cost_items(int H, int W) { return H * ((W + kXS - 1) / kXS); }
size_t cost_kernel_smem() { return cost_smem_bytes(); }

cudaError_t prepare_cost_batched()
{
    return fbs::raise_smem_limit(cost_batched_kernel, (int)cost_smem_bytes());
}

cudaError_t launch_stats_batched(const BatchPair* pairs, int npairs, int nitems, int* counter, int grid,
                                 cudaStream_t stream)
{
    fbs::note_launch();
    grey_stats_batched_kernel<<<grid, 256, 0, stream>>>(pairs, npairs, nitems, counter);
    return cudaGetLastError();
}

cudaError_t launch_cost_batched(const BatchPair* pairs, int npairs, int nitems, int* counter, int grid,
                                cudaStream_t stream)
{
    fbs::note_launch();
    cost_batched_kernel<<<grid, kThreads, cost_smem_bytes(), stream>>>(pairs, npairs, nitems, counter);
    return cudaGetLastError();
}

size_t cost_scratch_bytes(int H, int W)
{
    const size_t n = (size_t)2 * H * W;
    return ((n * sizeof(int16_t) + 255) & ~(size_t)255) + ((n * sizeof(int) + 255) & ~(size_t)255) +
           ((n * sizeof(float) + 255) & ~(size_t)255);
}

size_t rgbx_bytes(int H, int W) { return ((size_t)H * rgbx_pitch(W) * 8 + 255) & ~(size_t)255; }

__global__ void pack_rgbx_kernel(const uint8_t* __restrict__ img, int H, int W, int C, uint2* __restrict__ out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W) return;
    const uint8_t* p = img + ((size_t)y * W + x) * C;
    const uint32_t c = C == 3 ? (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) : (uint32_t)p[0];
    out[(size_t)y * rgbx_pitch(W) + x] = make_uint2(c, (uint32_t)__dp4a(c, c, 0u));
}

cudaError_t launch_pack_rgbx(const uint8_t* img, int H, int W, int C, uint2* rgbx, cudaStream_t stream)
{
    dim3 grid((W + 255) / 256, H);
    fbs::note_launch();
    pack_rgbx_kernel<<<grid, 256, 0, stream>>>(img, H, W, C, rgbx);
    return cudaGetLastError();
}

CostScratch carve_cost_scratch(void* base, int H, int W)
{
    const size_t n = (size_t)2 * H * W;
    CostScratch sc;
    sc.rgbx = nullptr;
    uint8_t* p = (uint8_t*)base;
    sc.g = (int16_t*)p;
    p += (n * sizeof(int16_t) + 255) & ~(size_t)255;
    sc.s = (int*)p;
    p += (n * sizeof(int) + 255) & ~(size_t)255;
    sc.rv = (float*)p;
    return sc;
}

cudaError_t launch_cost_build(const CostScratch& sc, const uint8_t* left, const uint8_t* right, int H, int W,
                              int C, int D, int ld, int mode, float tau, float* cost, cudaStream_t stream)
{
    if (mode == 0) {
        cudaError_t e = launch_stats(sc, left, right, H, W, C, stream);
        if (e != cudaSuccess) return e;
        return launch_cost_kernel<0, float>(sc, left, right, H, W, C, D, ld, tau, cost, stream);
    }
    return launch_cost_kernel<1, float>(sc, left, right, H, W, C, D, ld, tau, cost, stream);
}

cudaError_t launch_cost_band(const CostScratch& sc, const uint8_t* left, const uint8_t* right, int H, int W,
                             int C, int D, int ld, int radius, const int2* tile_range, float* cost, cudaStream_t stream)
{
    cudaError_t e = launch_stats(sc, left, right, H, W, C, stream);
    if (e != cudaSuccess) return e;
    const size_t smem = cost_smem_bytes();
    e = fbs::raise_smem_limit(cost_band_kernel, (int)smem);
    if (e != cudaSuccess) return e;
    const int ntx = (W + kAggTileX - 1) / kAggTileX, nty = (H + kAggTileY - 1) / kAggTileY;
    dim3 grid((W + kXS - 1) / kXS, H);
    fbs::note_launch();
    cost_band_kernel<<<grid, kThreads, smem, stream>>>(sc.g, sc.s, sc.rv, H, W, D, ld, radius, tile_range, ntx, nty,
                                                       cost);
    return cudaGetLastError();
}

cudaError_t launch_cost_build_lr(const CostScratch& sc, const uint8_t* left, const uint8_t* right, int H, int W,
                                 int C, int D, int ld, int mode, float tau, float* cost, float* cost_r,
                                 cudaStream_t stream)
{
    cudaError_t e = cudaSuccess;
    if (mode == 0) e = launch_stats(sc, left, right, H, W, C, stream);
    if (e != cudaSuccess) return e;
    const size_t smem = cost_smem_bytes();
    dim3 grid((W + kXS - 1) / kXS, H);
    if (mode == 0) {
        e = fbs::raise_smem_limit(cost_lr_kernel<0>, (int)smem);
        fbs::note_launch();
        if (e == cudaSuccess)
            cost_lr_kernel<0><<<grid, kThreads, smem, stream>>>(sc.g, sc.s, sc.rv, left, right, H, W, C, D, ld, tau,
                                                                cost, cost_r);
    } else {
        e = fbs::raise_smem_limit(cost_lr_kernel<1>, (int)smem);
        fbs::note_launch();
        if (e == cudaSuccess)
            cost_lr_kernel<1><<<grid, kThreads, smem, stream>>>(sc.g, sc.s, sc.rv, left, right, H, W, C, D, ld, tau,
                                                                cost, cost_r);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    fbs::note_launch();
    right_edge_fill_kernel<<<H, 256, 0, stream>>>(H, W, D, ld, mode == 0 ? 2.f : tau, cost_r);
    return cudaGetLastError();
}

cudaError_t launch_cost_build_xblock16(const CostScratch& sc, const uint8_t* left, const uint8_t* right, int H,
                                       int W, int C, int D, int mode, float tau, bool bf16, void* cost,
                                       cudaStream_t stream)
{
    // one launch: statistics, costs, pad rows and the packed guide (sc.rgbx)
    if (D > 256 || !sc.rgbx) return cudaErrorInvalidValue;   // serves the tensor-core form only
    if (mode == 0)
        return bf16 ? launch_cost_xb<0>(sc, left, right, H, W, C, D, tau, (__nv_bfloat16*)cost, stream)
                    : launch_cost_xb<0>(sc, left, right, H, W, C, D, tau, (__half*)cost, stream);
    return bf16 ? launch_cost_xb<1>(sc, left, right, H, W, C, D, tau, (__nv_bfloat16*)cost, stream)
                : launch_cost_xb<1>(sc, left, right, H, W, C, D, tau, (__half*)cost, stream);
}

}  // namespace fbs
