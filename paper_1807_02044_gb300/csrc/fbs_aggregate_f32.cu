// Steps 2-4 of fast bilateral stereo in FP32: bilateral aggregation of every
// disparity slice (Sec. II-B, Eq. (6)-(8)), winner-take-all (Sec. II-C) and
// the parabola refinement of Eq. (10) (Sec. II-D), in one kernel.
//
//   Agg(p, d) = sum_q w(p, q) C(q, d) / sum_q w(p, q),
//   w(p, q)   = exp(-|q - p|^2 / gamma_d^2) * exp(-|I(q) - I(p)|^2 / gamma_r^2),
// q over the (2 rho + 1)^2 window clipped to the image; I is the left image
// (for RGB the squared Euclidean colour distance).  The two exponentials are
// evaluated as one exp2 of the summed exponent.
//
// Work decomposition (one CTA = a 32 x 4 pixel tile and a chunk of DC
// disparities; 8 warps):
//   * Cost rows r = y0-rho .. y0+3+rho are streamed through a 3-deep ring of
//     shared-memory buffers with cp.async (zero-filled outside the image), and
//     the guide row r through a matching ring.
//   * For each streamed row, the CTA computes the weights w(p, q) of every
//     tile pixel p whose window contains row r -- once per (p, q), shared by
//     all DC disparities -- into a double-buffered shared array.
//   * Warp g owns tile columns 4g..4g+3; lane = (row yi, disparity group k).
//     A thread accumulates 4 pixels x KD disparities.  Along the window the
//     four cost columns it needs at tap dx are held in a rotating register
//     window, so each cost column is read from shared memory once and used
//     for up to 4 pixels, and each weight is a broadcast read used for KD
//     disparities.  Lanes of different rows read the same cost address
//     (broadcast), so a warp's cost read is one 128-byte wavefront.
//   * One __syncthreads per streamed row.
//   * After the last row the sums are normalised, staged in shared memory and
//     reduced per pixel: WTA with the smallest d on ties, plus the values at
//     d*-1 and d*+1 carried across chunks for Eq. (10).
#include "fbs_internal.cuh"

namespace fbs {
namespace {

constexpr int kTX = kAggTileX;   // tile width (pixels)
constexpr int kTY = kAggTileY;   // tile height (rows)
constexpr int kPX = 4;         // pixels per thread along x
constexpr int kThreads = 256;  // 8 warps
constexpr int kNPix = kTX * kTY;
// 2^23 as an FP32 bit pattern: for 0 <= c < 2^23 the pattern kMagic + c is the
// float 2^23 + c exactly.
constexpr uint32_t kMagic = 0x4B000000u;

__host__ __device__ inline int weight_stride(int rho)
{
    // per-row stride of the weight buffer [dx][kTX]; == 8 (mod 32) so that
    // the four rows of a warp read four different bank groups
    int n = (2 * rho + 1) * kTX;
    n = (n + 31) & ~31;
    return n + 8;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, int src_bytes)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <int DC>
__host__ __device__ inline size_t smem_bytes(int rho)
{
    const int NC = kTX + 2 * rho;
    const size_t ring = (size_t)3 * NC * DC;
    const size_t stage = (size_t)kNPix * (DC + 1);
    const size_t a = ring > stage ? ring : stage;
    return sizeof(float) * (a + 2 * (size_t)kTY * weight_stride(rho) + 2 * kNPix) + sizeof(uint2) * 3 * NC;
}

// Load cost row r, columns x0-rho .. x0-rho+NC-1, disparities dc0 .. dc0+DC-1;
// disparities >= D (the end of the range being aggregated) are zero-filled.
template <int DC, bool VEC>
__device__ __forceinline__ void load_cost_row(float* dst, const float* __restrict__ cost, int ld, int W,
                                              int D, int r, int x0, int rho, int NC, int dc0)
{
    if (VEC) {
        constexpr int NQ4 = DC / 4;
        for (int it = threadIdx.x; it < NC * NQ4; it += kThreads) {
            const int col = it / NQ4, q = it - col * NQ4;
            const int gx = x0 - rho + col;
            const int d = dc0 + 4 * q;
            const bool in = gx >= 0 && gx < W && d < D;
            const int gxc = in ? gx : 0;
            const int dcl = in ? d : 0;
            const float* src = cost + ((size_t)r * W + gxc) * ld + dcl;
            const int bytes = in ? 4 * min(4, D - d) : 0;
            cp_async16(dst + col * DC + 4 * q, src, bytes);
        }
    } else {
        for (int it = threadIdx.x; it < NC * DC; it += kThreads) {
            const int col = it / DC, q = it - col * DC;
            const int gx = x0 - rho + col;
            const int d = dc0 + q;
            const bool in = gx >= 0 && gx < W && d < D;
            const float* src = cost + ((size_t)r * W + (in ? gx : 0)) * ld + (in ? d : 0);
            cp_async4(dst + col * DC + q, src, in ? 4 : 0);
        }
    }
}

// A guide pixel as (R | G << 8 | B << 16, R^2 + G^2 + B^2); grey images use
// the first channel only.
__device__ __forceinline__ uint2 packed_colour(const uint8_t* p, int C)
{
    const uint32_t c = C == 3 ? (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) : (uint32_t)p[0];
    return make_uint2(c, (uint32_t)__dp4a(c, c, 0u));
}

__device__ __forceinline__ void load_guide_row(uint2* dst, const uint8_t* __restrict__ guide, int W, int C, int r,
                                               int x0, int rho, int NC)
{
    for (int col = threadIdx.x; col < NC; col += kThreads) {
        const int gx = x0 - rho + col;
        dst[col] = (gx >= 0 && gx < W) ? packed_colour(guide + ((size_t)r * W + gx) * C, C) : make_uint2(0u, 0u);
    }
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// One 32 x 4 tile with top-left pixel (x0, y0), disparities [d_begin, d_end)
// (the full range: 0, D); ends with a __syncthreads, so a CTA may call it for
// several tiles in a row.  band (nullable) restricts the WTA and Eq. (10) of
// each pixel to its own band [lo, hi], a sub-range of [d_begin, d_end);
// without it every pixel uses [0, D-1].  d_begin must be a multiple of 4.
template <int KD, bool VEC>
__device__ __forceinline__ void aggregate_tile(const float* __restrict__ cost, int ld,
                                               const uint8_t* __restrict__ guide, int H, int W, int C, int D,
                                               int rho, float neg_ks, float neg_kr, float* __restrict__ agg_out,
                                               int32_t* __restrict__ disp_int, float* __restrict__ disp_sub, int x0,
                                               int y0, float4* smem_f4, int d_begin, int d_end,
                                               const uint32_t* __restrict__ band)
{
    constexpr int DC = 8 * KD;   // disparities per chunk
    constexpr int NQ = KD / 4;   // float4 groups per thread

    const int tid = threadIdx.x;
    const int lane = tid & 31, g = tid >> 5;
    const int yi = lane >> 3, k = lane & 7;
    const int NC = kTX + 2 * rho;
    const int NT = 2 * rho + 1;
    const int WS = weight_stride(rho);

    // shared memory: guide ring [3][NC] uint2 | cost ring [3][NC][DC] (aliased
    // by the stage [kNPix][DC+1]) | weights [2][kTY][WS] | den [2][kNPix].  NC
    // is even, so the cost ring starts 16-byte aligned.
    uint2* const gring = (uint2*)smem_f4;
    float* const cring = (float*)(gring + 3 * NC);
    float* const stage = cring;
    const int cslot = NC * DC;
    const int ring_sz = 3 * NC * DC, stage_sz = kNPix * (DC + 1);
    float* const wring = cring + (ring_sz > stage_sz ? ring_sz : stage_sz);
    const int wslot = kTY * WS;
    float* const den_s = wring + 2 * wslot;

    // producer role: pixel pp of the tile, half of the dx range
    const int pp = tid & (kNPix - 1);
    const int half = tid >> 7;
    const int pyi = pp / kTX, ppx = pp % kTX;
    const int py = y0 + pyi, pxg = x0 + ppx;
    const bool pvalid = py < H && pxg < W;
    const int dx_lo = half ? rho + 1 : 0;
    const int dx_hi = half ? NT : rho + 1;
    // the pixel's colour and |p|^2 + 2^23 (so |q - p|^2 = |q|^2 + |p|^2 - 2 q.p,
    // exact in integers and below 2^23, becomes the bit pattern of 2^23 + c)
    uint32_t pcol = 0u, pnorm = kMagic;
    if (pvalid) {
        const uint2 c = packed_colour(guide + ((size_t)py * W + pxg) * C, C);
        pcol = c.x;
        pnorm = c.y + kMagic;
    }

    // WTA role (tid < kNPix): state of pixel tid carried across chunks
    float best = __int_as_float(0x7f800000), a_prev = 0.f, a_next = 0.f, last = 0.f;
    int blo = 0, bhi = D - 1;
    // Disparity range of each 4-column group (the pixels of one consumer
    // warp): the union of its pixels' bands.  A warp skips the chunks outside
    // its range, and the weights of its pixels are not generated for them.
    __shared__ int grp_lo[kTX / kPX], grp_hi[kTX / kPX];
    if (band != nullptr) {
        if (tid < kTX / kPX) {
            grp_lo[tid] = D;
            grp_hi[tid] = -1;
        }
        __syncthreads();
        if (tid < kNPix) {
            const int oy = y0 + tid / kTX, ox = x0 + tid % kTX;
            if (oy < H && ox < W) {
                const uint32_t b = band[(size_t)oy * W + ox];
                blo = (int)(b & 0xffffu);
                bhi = (int)(b >> 16);
                atomicMin(&grp_lo[(tid % kTX) / kPX], blo);
                atomicMax(&grp_hi[(tid % kTX) / kPX], bhi);
            }
        }
        __syncthreads();
    }
    int bidx = blo;
    bool pending = false;

    // consumer role
    const int y = y0 + yi;
    const int r_lo = max(0, y0 - rho);
    const int r_hi = min(H - 1, y0 + kTY - 1 + rho);
    const int nr = r_hi - r_lo + 1;

    for (int dc0 = d_begin; dc0 < d_end; dc0 += DC) {
        // this chunk is needed by the producer's pixel group / the consumer's group
        const bool p_on = band == nullptr || (grp_hi[ppx / kPX] >= dc0 && grp_lo[ppx / kPX] < dc0 + DC);
        const bool c_on = band == nullptr || (grp_hi[g] >= dc0 && grp_lo[g] < dc0 + DC);
        float4 acc[kPX][NQ];
#pragma unroll
        for (int i = 0; i < kPX; ++i)
#pragma unroll
            for (int q = 0; q < NQ; ++q) acc[i][q] = make_float4(0.f, 0.f, 0.f, 0.f);
        float den_part = 0.f;

        load_cost_row<DC, VEC>(cring, cost, ld, W, d_end, r_lo, x0, rho, NC, dc0);
        cp_async_commit();
        load_guide_row(gring, guide, W, C, r_lo, x0, rho, NC);
        __syncthreads();

        for (int s = 0; s < nr; ++s) {
            const int r = r_lo + s;
            // (A) prefetch the next cost row, (B) the next guide row
            if (s + 1 < nr) {
                load_cost_row<DC, VEC>(cring + ((s + 1) % 3) * cslot, cost, ld, W, d_end, r + 1, x0, rho, NC, dc0);
                load_guide_row(gring + ((s + 1) % 3) * NC, guide, W, C, r + 1, x0, rho, NC);
            }
            cp_async_commit();
            // (C) weights of row r for every tile pixel whose window reaches it
            {
                const int dy = r - py;
                if (p_on && py < H && dy >= -rho && dy <= rho) {
                    const uint2* gr = gring + (s % 3) * NC;
                    float* wrow = wring + (s & 1) * wslot + pyi * WS;
                    const int dy2 = dy * dy;
                    for (int dx = dx_lo; dx < dx_hi; ++dx) {
                        const int qx = pxg + dx - rho;
                        float w = 0.f;
                        if (pxg < W && qx >= 0 && qx < W) {
                            // Eq. (7)-(8) as one exp2: colour distance exact in
                            // integers, then float(c) = (2^23 + c) - 2^23 exactly
                            const uint2 q = gr[ppx + dx];
                            const float col2 =
                                __uint_as_float(q.y + pnorm - 2u * (uint32_t)__dp4a(q.x, pcol, 0u)) - 8388608.f;
                            const int ddx = dx - rho;
                            const float sp2 = (float)(ddx * ddx + dy2);
                            w = ex2_approx(fmaf(col2, neg_kr, sp2 * neg_ks));
                        }
                        wrow[dx * kTX + ppx] = w;
                        den_part += w;
                    }
                }
            }
            // (D) own copies of row r have landed; (E) everyone's have
            cp_async_wait1();
            __syncthreads();
            // (F) accumulate row r
            const int dy = r - y;
            if (c_on && y < H && dy >= -rho && dy <= rho) {
                const float* cr = cring + (s % 3) * cslot + (kPX * g) * DC + 4 * k;
                const float* wr = wring + (s & 1) * wslot + yi * WS + kPX * g;
                float4 win[4][NQ];
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int q = 0; q < NQ; ++q) win[j][q] = *(const float4*)(cr + j * DC + 32 * q);
                for (int dx0 = 0; dx0 < NT; dx0 += 4) {
#pragma unroll
                    for (int s4 = 0; s4 < 4; ++s4) {
                        const int dx = dx0 + s4;
                        if (dx < NT) {
#pragma unroll
                            for (int q = 0; q < NQ; ++q)
                                win[(s4 + 3) & 3][q] = *(const float4*)(cr + (dx + 3) * DC + 32 * q);
                            const float4 w4 = *(const float4*)(wr + dx * kTX);
                            const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                            for (int i = 0; i < kPX; ++i) {
                                const int slot = (i + s4) & 3;
#pragma unroll
                                for (int q = 0; q < NQ; ++q) {
                                    acc[i][q].x = fmaf(wv[i], win[slot][q].x, acc[i][q].x);
                                    acc[i][q].y = fmaf(wv[i], win[slot][q].y, acc[i][q].y);
                                    acc[i][q].z = fmaf(wv[i], win[slot][q].z, acc[i][q].z);
                                    acc[i][q].w = fmaf(wv[i], win[slot][q].w, acc[i][q].w);
                                }
                            }
                        }
                    }
                }
            }
        }

        // normalise and stage: stage[pixel][d] with pixel = yi*kTX + 4g + i
        den_s[half * kNPix + pp] = den_part;
        __syncthreads();   // all rows consumed, ring free; den visible
#pragma unroll
        for (int i = 0; i < kPX; ++i) {
            const int pix = yi * kTX + kPX * g + i;
            const float den = den_s[pix] + den_s[kNPix + pix];
            const float inv = 1.f / den;
            float* st = stage + pix * (DC + 1) + 4 * k;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                st[32 * q + 0] = acc[i][q].x * inv;
                st[32 * q + 1] = acc[i][q].y * inv;
                st[32 * q + 2] = acc[i][q].z * inv;
                st[32 * q + 3] = acc[i][q].w * inv;
            }
        }
        __syncthreads();
        const int nd = min(DC, d_end - dc0);
        if (agg_out != nullptr) {
            for (int e = tid; e < kNPix * nd; e += kThreads) {
                const int pix = e / nd, j = e - pix * nd;
                const int ey = y0 + pix / kTX, ex = x0 + pix % kTX;
                if (ey < H && ex < W) agg_out[((size_t)ey * W + ex) * D + dc0 + j] = stage[pix * (DC + 1) + j];
            }
        }
        if (tid < kNPix) {
            const float* st = stage + tid * (DC + 1);
            const int j0 = max(0, blo - dc0), j1 = min(nd, bhi + 1 - dc0);
            for (int j = j0; j < j1; ++j) {
                const float v = st[j];
                if (pending) {
                    a_next = v;
                    pending = false;
                }
                if (v < best) {
                    best = v;
                    bidx = dc0 + j;
                    a_prev = last;
                    pending = true;
                }
                last = v;
            }
        }
        __syncthreads();   // stage (aliasing the ring) consumed before the next chunk reloads it
    }

    if (tid < kNPix) {
        const int oy = y0 + tid / kTX, ox = x0 + tid % kTX;
        if (oy < H && ox < W) {
            float ds = (float)bidx;
            if (bidx > blo && bidx < bhi) {
                const float den = 2.f * a_prev + 2.f * a_next - 4.f * best;
                if (den > 0.f) ds = (float)bidx + (a_prev - a_next) / den;
            }
            const size_t o = (size_t)oy * W + ox;
            if (disp_int) disp_int[o] = bidx;
            if (disp_sub) disp_sub[o] = ds;
        }
    }
}

template <int KD, bool VEC>
__global__ void __launch_bounds__(kThreads, 2)
aggregate_f32_kernel(const float* __restrict__ cost, int ld, const uint8_t* __restrict__ guide, int H,
                     int W, int C, int D, int rho, float neg_ks, float neg_kr,
                     float* __restrict__ agg_out, int32_t* __restrict__ disp_int,
                     float* __restrict__ disp_sub)
{
    extern __shared__ float4 smem_f4[];
    aggregate_tile<KD, VEC>(cost, ld, guide, H, W, C, D, rho, neg_ks, neg_kr, agg_out, disp_int, disp_sub,
                            blockIdx.x * kTX, blockIdx.y * kTY, smem_f4, 0, D, nullptr);
}

// Band form: tile t aggregates its range tile_range[t] (chunks of 32 or 64
// disparities) and each pixel takes its winner inside its own band.
__global__ void __launch_bounds__(kThreads, 2)
aggregate_band_kernel(const float* __restrict__ cost, int ld, const uint8_t* __restrict__ guide, int H, int W,
                      int C, int D, int rho, float neg_ks, float neg_kr, const int2* __restrict__ tile_range,
                      const uint32_t* __restrict__ band, int32_t* __restrict__ disp_int,
                      float* __restrict__ disp_sub)
{
    extern __shared__ float4 smem_f4[];
    const int2 r = tile_range[(size_t)blockIdx.y * gridDim.x + blockIdx.x];
    if (r.y - r.x > 32)
        aggregate_tile<8, true>(cost, ld, guide, H, W, C, D, rho, neg_ks, neg_kr, nullptr, disp_int, disp_sub,
                                blockIdx.x * kTX, blockIdx.y * kTY, smem_f4, r.x, r.y, band);
    else
        aggregate_tile<4, true>(cost, ld, guide, H, W, C, D, rho, neg_ks, neg_kr, nullptr, disp_int, disp_sub,
                                blockIdx.x * kTX, blockIdx.y * kTY, smem_f4, r.x, r.y, band);
}

// Persistent form over a batch: CTAs claim (pair, tile) items from a counter;
// pairs[p].agg_off is the first item of pair p, items of a pair are its tiles
// in row-major order.  No CTA waits on another.
__global__ void __launch_bounds__(kThreads, 2)
aggregate_f32_batched_kernel(const BatchPair* __restrict__ pairs, int npairs, int nitems, int* __restrict__ counter)
{
    extern __shared__ float4 smem_f4[];
    __shared__ int item_s;
    for (;;) {
        if (threadIdx.x == 0) item_s = atomicAdd(counter, 1);
        __syncthreads();
        const int item = item_s;
        __syncthreads();
        if (item >= nitems) break;
        const int pi = find_pair(pairs, npairs, item, &BatchPair::agg_off);
        const BatchPair& bp = pairs[pi];
        const int t = item - bp.agg_off;
        const int ntx = (bp.W + kTX - 1) / kTX;
        aggregate_tile<8, true>(bp.cost, bp.ld, bp.left, bp.H, bp.W, bp.C, bp.D, bp.radius, bp.neg_ks, bp.neg_kr,
                                nullptr, bp.disp_int, bp.disp_sub, (t % ntx) * kTX, (t / ntx) * kTY, smem_f4, 0,
                                bp.D, nullptr);
    }
}

template <int KD, bool VEC>
cudaError_t launch_kd(const float* cost, int ld, const uint8_t* guide, int H, int W, int C, int D,
                      int rho, float neg_ks, float neg_kr, float* agg_out, int32_t* disp_int,
                      float* disp_sub, cudaStream_t stream)
{
    const size_t smem = smem_bytes<8 * KD>(rho);
    cudaError_t e = fbs::raise_smem_limit(aggregate_f32_kernel<KD, VEC>, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((W + kTX - 1) / kTX, (H + kTY - 1) / kTY);
    fbs::note_launch();
    aggregate_f32_kernel<KD, VEC><<<grid, kThreads, smem, stream>>>(
        cost, ld, guide, H, W, C, D, rho, neg_ks, neg_kr, agg_out, disp_int, disp_sub);
    return cudaGetLastError();
}

}  // namespace

int agg_f32_tiles(int H, int W) { return ((W + kTX - 1) / kTX) * ((H + kTY - 1) / kTY); }

cudaError_t prepare_aggregate_f32_batched(int max_radius, size_t* smem_out)
{
    const size_t smem = smem_bytes<64>(max_radius);
    *smem_out = smem;
    return fbs::raise_smem_limit(aggregate_f32_batched_kernel, (int)smem);
}

cudaError_t launch_aggregate_f32_batched(const BatchPair* pairs, int npairs, int nitems, int* counter, int grid,
                                         size_t smem, cudaStream_t stream)
{
    fbs::note_launch();
    aggregate_f32_batched_kernel<<<grid, kThreads, smem, stream>>>(pairs, npairs, nitems, counter);
    return cudaGetLastError();
}

cudaError_t launch_aggregate_band(const float* cost, int ld, const uint8_t* guide, int H, int W, int C, int D,
                                  int radius, float sigma_s, float sigma_r, const int2* tile_range,
                                  const uint32_t* band, int32_t* disp_int, float* disp_sub, cudaStream_t stream)
{
    const double log2e = 1.4426950408889634;
    const float neg_ks = (float)(-log2e / ((double)sigma_s * sigma_s));
    const float neg_kr = (float)(-log2e / ((double)sigma_r * sigma_r));
    const size_t smem = smem_bytes<64>(radius);
    cudaError_t e = fbs::raise_smem_limit(aggregate_band_kernel, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((W + kTX - 1) / kTX, (H + kTY - 1) / kTY);
    fbs::note_launch();
    aggregate_band_kernel<<<grid, kThreads, smem, stream>>>(cost, ld, guide, H, W, C, D, radius, neg_ks, neg_kr,
                                                            tile_range, band, disp_int, disp_sub);
    return cudaGetLastError();
}

cudaError_t launch_aggregate_f32(const float* cost, int ld, const uint8_t* guide, int H, int W, int C,
                                 int D, int radius, float sigma_s, float sigma_r, float* agg_out,
                                 int32_t* disp_int, float* disp_sub, cudaStream_t stream)
{
    // exp(-a/g^2) = exp2(-a * log2(e) / g^2)
    const double log2e = 1.4426950408889634;
    const float neg_ks = (float)(-log2e / ((double)sigma_s * sigma_s));
    const float neg_kr = (float)(-log2e / ((double)sigma_r * sigma_r));
    const bool vec = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(cost) & 15) == 0);
    if (D <= 32) {
        return vec ? launch_kd<4, true>(cost, ld, guide, H, W, C, D, radius, neg_ks, neg_kr, agg_out, disp_int, disp_sub, stream)
                   : launch_kd<4, false>(cost, ld, guide, H, W, C, D, radius, neg_ks, neg_kr, agg_out, disp_int, disp_sub, stream);
    }
    return vec ? launch_kd<8, true>(cost, ld, guide, H, W, C, D, radius, neg_ks, neg_kr, agg_out, disp_int, disp_sub, stream)
               : launch_kd<8, false>(cost, ld, guide, H, W, C, D, radius, neg_ks, neg_kr, agg_out, disp_int, disp_sub, stream);
}

}  // namespace fbs
