// Kernels of the band-proposal network: 3x3 convolutions and weight gradients
// on the tensor cores (forward, data gradient, weight gradient), loss, Adam and
// the packing of FP32 master weights into BF16 MMA operands.
//
// Convolution as an implicit GEMM (one CTA = 128 consecutive quarter pixels
// = the MMA's M; persistent over tiles):
//     out[m][n] = sum_k A[m][k] B[n][k],   k = (tap, channel),
//     A[m][k]   = in[pixel m shifted by tap][channel]  (zero outside the image),
//     B[n][k]   = W[tap][channel][n]  (forward)  or  W[tap][n][channel]  (data
//                 gradient, with the tap offsets negated).
// Both operands are K-major core matrices in shared memory (8 rows x 16 bytes;
// LBO = distance between core matrices along K, SBO = 128 bytes between row
// groups).  Every thread gathers its pixel's row of A with 16-byte loads (one
// load = 8 channels of one tap = one core-matrix row) and stores it with
// 16-byte shared stores; one thread issues the K/16 tcgen05.mma of the tile
// into a TMEM accumulator (M = 128 lanes x N columns, FP32) and commits to an
// mbarrier; the four warps then read their 32 lanes back (tcgen05.ld), apply
// the epilogue and store.  The weight image (B) is loaded once per CTA.
// Every mbarrier wait is bounded; a timeout sets the error word, and all
// threads leave the tile loop together, free the tensor memory and return.
#include <cuda_bf16.h>

#include "fbs_band_net.cuh"
#include "fbs_internal.cuh"
#include "tc_ptx.cuh"

namespace fbs {
namespace bnet {
namespace {

using namespace tc;

constexpr int kConvThreads = 128;
constexpr int kM = 128;

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

template <int CIN, int N>
__global__ void __launch_bounds__(kConvThreads)
conv3x3_tc_kernel(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ image,
                  const float* __restrict__ bias, const __nv_bfloat16* __restrict__ mask, void* __restrict__ out,
                  int nout, int Hq, int Wq, int flip, int mode, int* __restrict__ err)
{
    constexpr int KC = k_cores(CIN);            // core matrices along K
    constexpr int KREAL = 9 * CIN / 8;          // of which hold data
    constexpr int A_BYTES = KC * kM * 16;
    constexpr int B_BYTES = KC * N * 16;
    constexpr int CH = CIN / 8;                 // 16-byte chunks per (pixel, tap)
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t* As = sm;
    uint8_t* Bs = sm + A_BYTES;
    uint64_t* bar = reinterpret_cast<uint64_t*>(Bs + B_BYTES);
    uint32_t* misc = reinterpret_cast<uint32_t*>(bar + 1);   // [0] TMEM address, [1] abort flag

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int P = Hq * Wq;
    const int ntiles = (P + kM - 1) / kM;

    for (int i = tid; i < B_BYTES / 16; i += kConvThreads)
        reinterpret_cast<uint4*>(Bs)[i] = reinterpret_cast<const uint4*>(image)[i];
    for (int kc = KREAL; kc < KC; ++kc) reinterpret_cast<uint4*>(As + kc * kM * 16)[tid] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        mbar_init(smem_u32(bar), 1);
        misc[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_u32(&misc[0]), 32);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = misc[0];
    const uint32_t idesc = idesc_f16(true, kM, N);
    const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);

    uint32_t phase = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        // ---- gather this thread's row of A -------------------------------
        const int p = tile * kM + tid;
        const int Y = p / Wq, X = p - Y * Wq;
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            int dy = t / 3 - 1, dx = t % 3 - 1;
            if (flip) {
                dy = -dy;
                dx = -dx;
            }
            const int yy = Y + dy, xx = X + dx;
            const bool ok = p < P && yy >= 0 && yy < Hq && xx >= 0 && xx < Wq;
            const uint4* src = reinterpret_cast<const uint4*>(in + ((size_t)(ok ? yy * Wq + xx : 0)) * CIN);
#pragma unroll
            for (int j = 0; j < CH; ++j) {
                const uint4 v = ok ? src[j] : make_uint4(0, 0, 0, 0);
                *reinterpret_cast<uint4*>(As + ((t * CH + j) * kM + tid) * 16) = v;
            }
        }
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        // ---- one thread issues the tile's MMAs ----------------------------
        if (tid == 0) {
            tc_fence_after();
#pragma unroll 1
            for (int ks = 0; ks < KC / 2; ++ks) {
                const uint64_t ad = sdesc(a0 + ks * 2 * kM * 16, kM * 16, 128);
                const uint64_t bd = sdesc(b0 + ks * 2 * N * 16, N * 16, 128);
                umma_f16(tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
            }
            umma_commit(smem_u32(bar));
        }
        const bool ok = mbar_wait(smem_u32(bar), phase);
        phase ^= 1u;
        if (!ok) atomicExch(&misc[1], 1u);
        tc_fence_before();
        __syncthreads();
        if (misc[1] != 0) {
            if (tid == 0) {
                atomicCAS(err, 0, 21);
                mbar_wait(smem_u32(bar), phase ^ 1u);   // once more, bounded, for the MMAs in flight
            }
            break;
        }
        tc_fence_after();
        // ---- epilogue: warp w holds TMEM lanes 32w .. 32w+31 ---------------
        float v[N];
#pragma unroll
        for (int c = 0; c < N; c += 16) {
            float t16[16];
            tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, t16);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[c + i] = t16[i];
        }
        const int po = tile * kM + 32 * warp + lane;
        if (po < P) {
            if (mode == kConvLinearF32) {
                float* o = reinterpret_cast<float*>(out) + (size_t)po * nout;
#pragma unroll
                for (int c = 0; c < N; ++c)
                    if (c < nout) o[c] = v[c] + bias[c];
            } else {
                if (mode == kConvReluBf16) {
#pragma unroll
                    for (int c = 0; c < N; ++c) v[c] = fmaxf(v[c] + bias[c], 0.f);
                } else {
                    const uint4* mk = reinterpret_cast<const uint4*>(mask + (size_t)po * N);
#pragma unroll
                    for (int q = 0; q < N / 8; ++q) {
                        const uint4 w = mk[q];
                        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            // a BF16 value is > 0 iff its sign bit is clear and it is not +0
                            const uint32_t lo = ws[h] & 0xffffu, hi = ws[h] >> 16;
                            if (lo == 0u || (lo & 0x8000u)) v[8 * q + 2 * h] = 0.f;
                            if (hi == 0u || (hi & 0x8000u)) v[8 * q + 2 * h + 1] = 0.f;
                        }
                    }
                }
                uint4* o = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(out) + (size_t)po * N);
#pragma unroll
                for (int q = 0; q < N / 8; ++q)
                    o[q] = make_uint4(pack_bf16x2(v[8 * q], v[8 * q + 1]), pack_bf16x2(v[8 * q + 2], v[8 * q + 3]),
                                      pack_bf16x2(v[8 * q + 4], v[8 * q + 5]), pack_bf16x2(v[8 * q + 6], v[8 * q + 7]));
            }
        }
        tc_fence_before();
        __syncthreads();   // A and the accumulator are free for the next tile
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 32);
}

template <int CIN, int N>
cudaError_t launch_conv_t(const __nv_bfloat16* in, const __nv_bfloat16* image, const float* bias,
                          const __nv_bfloat16* mask, void* out, int nout, int Hq, int Wq, int flip, int mode, int* err,
                          int num_sms, cudaStream_t stream)
{
    constexpr int KC = k_cores(CIN);
    const size_t smem = (size_t)KC * kM * 16 + (size_t)KC * N * 16 + 16;
    cudaError_t e = fbs::raise_smem_limit(conv3x3_tc_kernel<CIN, N>, (int)smem);
    if (e != cudaSuccess) return e;
    const int ntiles = (Hq * Wq + kM - 1) / kM;
    const int grid = ntiles < 2 * num_sms ? ntiles : 2 * num_sms;
    fbs::note_launch();
    conv3x3_tc_kernel<CIN, N><<<grid, kConvThreads, smem, stream>>>(in, image, bias, mask, out, nout, Hq, Wq, flip,
                                                                    mode, err);
    return cudaGetLastError();
}

// ---- weight gradients on the tensor cores ---------------------------------------
// dW[(t, ci)][co] = sum_p X[p + off(t)][ci] G[p][co] and the bias gradient
// sum_p G[p][co] as one product D[M][N] += A[M][K] B[N][K] with K = pixels: A
// row t * CIN + ci holds X[p + off(t)][ci] over the pixels p of a chunk (zero
// where p + off(t) leaves the image), row 9 CIN is all ones (its result is the
// bias gradient) and the rest zero; B row co holds G[p][co].  X and G are
// pixel-major in memory, so a warp loads an 8-pixel x 8-channel block (4 bytes
// per lane), transposes it in registers (movmatrix) and stores it as one
// K-major core matrix -- the operand layout of the convolutions above.  A CTA
// accumulates its chunks in TMEM (M-tiles of 128 rows) and writes one
// partial; wgrad_reduce_kernel adds the partials in a fixed order.
constexpr int kWgChunk = 128;        // pixels (K) per chunk
constexpr int kWgThreads = 256;

__device__ __forceinline__ uint32_t movmatrix_trans(uint32_t a)
{
    uint32_t d;
    asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(d) : "r"(a));
    return d;
}

template <int CIN, int COUT>
struct WgShape {
    static constexpr int MR = 9 * CIN + 1;                 // rows in use: taps x channels, ones
    static constexpr int MT = (MR + kM - 1) / kM;          // M-tiles of 128 rows
    static constexpr int N = COUT < 16 ? 16 : COUT;        // MMA N (a multiple of 16 for M = 128)
    static constexpr int KB = kWgChunk / 8;                // core matrices along K per chunk
    static constexpr uint32_t LBO_A = MT * kM * 16, LBO_B = N * 16;
    static constexpr int A_BYTES = KB * LBO_A, B_BYTES = KB * LBO_B;
    static constexpr uint32_t TMEM_COLS = MT * N <= 32 ? 32 : MT * N <= 64 ? 64 : MT * N <= 128 ? 128 : 256;
    static constexpr size_t SMEM = (size_t)A_BYTES + B_BYTES + 16;
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(kWgThreads)
wgrad_tc_kernel(const __nv_bfloat16* __restrict__ X, const __nv_bfloat16* __restrict__ G, int Hq, int Wq,
                float* __restrict__ partial, int* __restrict__ err)
{
    using S = WgShape<CIN, COUT>;
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t* As = sm;
    uint8_t* Bs = sm + S::A_BYTES;
    uint64_t* bar = reinterpret_cast<uint64_t*>(Bs + S::B_BYTES);
    uint32_t* misc = reinterpret_cast<uint32_t*>(bar + 1);   // [0] TMEM address, [1] abort flag
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int P = Hq * Wq;
    const int nchunks = (P + kWgChunk - 1) / kWgChunk;

    // rows 9 CIN .. of A (the ones row, then zeros) and rows COUT .. of B never
    // change: one 16-byte core-matrix row per store
    constexpr int ROWS_FIXED = S::MT * kM - 9 * CIN;
    const uint4 ones = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
    for (int i = tid; i < S::KB * ROWS_FIXED; i += kWgThreads) {
        const int kb = i / ROWS_FIXED, r = 9 * CIN + i - kb * ROWS_FIXED;
        *reinterpret_cast<uint4*>(As + kb * S::LBO_A + r * 16) = r == 9 * CIN ? ones : make_uint4(0u, 0u, 0u, 0u);
    }
    if constexpr (S::N > COUT) {
        for (int i = tid; i < S::KB * (S::N - COUT); i += kWgThreads) {
            const int kb = i / (S::N - COUT), r = COUT + i - kb * (S::N - COUT);
            *reinterpret_cast<uint4*>(Bs + kb * S::LBO_B + r * 16) = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    if (tid == 0) {
        mbar_init(smem_u32(bar), 1);
        misc[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_u32(&misc[0]), S::TMEM_COLS);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = misc[0];
    const uint32_t idesc = idesc_f16(true, kM, S::N);
    const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
    // lane -> (pixel of the 8-pixel group, channel pair of the 8-channel group),
    // the movmatrix fragment of the [pixel][channel] block; after the
    // transpose the lane holds channel lane/4 for pixels 2 (lane%4), + 1
    const int lp = lane >> 2, lc = 2 * (lane & 3);

    uint32_t phase = 0;
    bool first = true, aborted = false;
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int p0 = c * kWgChunk;
        // a warp fills the K columns of one 8-pixel group at a time: each lane
        // locates its pixel once, then loads every tap and channel group
        constexpr int CG = CIN / 8;
        for (int pg = warp; pg < S::KB; pg += kWgThreads / 32) {
            const int p = p0 + pg * 8 + lp;
            const bool pin = p < P;
            const int Y = pin ? p / Wq : 0, Xp = pin ? p - Y * Wq : 0;
            uint8_t* arow = As + pg * S::LBO_A + lp * 16 + 2 * lc;
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const int yy = Y + t / 3 - 1, xx = Xp + t % 3 - 1;
                const bool ok = pin && yy >= 0 && yy < Hq && xx >= 0 && xx < Wq;
                const __nv_bfloat16* src = X + (size_t)(ok ? yy * Wq + xx : 0) * CIN + lc;
                uint32_t v[CG];
#pragma unroll
                for (int cg = 0; cg < CG; ++cg) v[cg] = ok ? *reinterpret_cast<const uint32_t*>(src + cg * 8) : 0u;
#pragma unroll
                for (int cg = 0; cg < CG; ++cg)
                    *reinterpret_cast<uint32_t*>(arow + (t * CIN + cg * 8) * 16) = movmatrix_trans(v[cg]);
            }
            uint8_t* brow = Bs + pg * S::LBO_B + lp * 16 + 2 * lc;
#pragma unroll
            for (int cg = 0; cg < COUT / 8; ++cg) {
                const uint32_t v = pin ? *reinterpret_cast<const uint32_t*>(G + (size_t)p * COUT + cg * 8 + lc) : 0u;
                *reinterpret_cast<uint32_t*>(brow + cg * 8 * 16) = movmatrix_trans(v);
            }
        }
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll 1
            for (int m = 0; m < S::MT; ++m)
#pragma unroll 1
                for (int ks = 0; ks < S::KB / 2; ++ks) {
                    const uint64_t ad = sdesc(a0 + m * kM * 16 + ks * 2 * S::LBO_A, S::LBO_A, 128);
                    const uint64_t bd = sdesc(b0 + ks * 2 * S::LBO_B, S::LBO_B, 128);
                    umma_f16(tmem + (uint32_t)(m * S::N), ad, bd, idesc, (first && ks == 0) ? 0u : 1u);
                }
            umma_commit(smem_u32(bar));
        }
        const bool ok = mbar_wait(smem_u32(bar), phase);
        phase ^= 1u;
        if (!ok) atomicExch(&misc[1], 1u);
        tc_fence_before();
        __syncthreads();   // A and B are free for the next chunk
        if (misc[1] != 0) {
            if (tid == 0) {
                atomicCAS(err, 0, 22);
                mbar_wait(smem_u32(bar), phase ^ 1u);   // once more, bounded, for the MMAs in flight
            }
            aborted = true;
            break;
        }
        first = false;
    }
    if (!aborted && !first) {
        // warp w reads TMEM lanes 32w .. 32w+31 of every M-tile: A rows m*128 + 32w + lane
        tc_fence_after();
        float* part = partial + (size_t)blockIdx.x * (9 * CIN * COUT + COUT);
#pragma unroll 1
        for (int m = 0; m < S::MT; ++m) {
            const int r = m * kM + 32 * warp + lane;
#pragma unroll
            for (int cb = 0; cb < S::N; cb += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(m * S::N + cb), v);
                if (r < S::MR) {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (cb + i < COUT) part[r * COUT + cb + i] = v[i];
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, S::TMEM_COLS);
}

// grad[layer l] = sum over the nblk partials, dropping padded channels.
__global__ void wgrad_reduce_kernel(const float* __restrict__ partial, int nblk, int stride, int cinp, int coutp,
                                    int ci_real, int co_real, float* __restrict__ grad)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= stride) return;
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * stride + j];
    const int nw = 9 * cinp * coutp;
    if (j < nw) {
        const int t = j / (cinp * coutp), r = j % (cinp * coutp);
        const int ci = r / coutp, co = r % coutp;
        if (ci < ci_real && co < co_real) grad[(t * ci_real + ci) * co_real + co] = s;
    } else {
        const int co = j - nw;
        if (co < co_real) grad[9 * ci_real * co_real + co] = s;
    }
}

// ---- loss ------------------------------------------------------------------------
constexpr int kLossThreads = 256;

__global__ void __launch_bounds__(kLossThreads)
loss_kernel(const float* __restrict__ out, const int32_t* __restrict__ estar, const int32_t* __restrict__ label_int,
            const float* __restrict__ label_sub, int H, int W, int D, int h, __nv_bfloat16* __restrict__ G6,
            float* __restrict__ loss_partial)
{
    const int Hq = (H + 3) / 4, Wq = (W + 3) / 4, P = Hq * Wq;
    const int i = blockIdx.x * kLossThreads + threadIdx.x;
    float li = 0.f;
    if (i < P) {
        const int Y = i / Wq, X = i - Y * Wq;
        const float o0 = out[2 * i], z = out[2 * i + 1];
        const float c = __fmul_rn(4.f, __fadd_rn((float)estar[i], o0));
        float m = floorf(__fadd_rn(c, 0.5f));
        if (!(m >= 0.f)) m = 0.f;
        if (m > (float)(D - 1)) m = (float)(D - 1);
        const int mi = (int)m;
        // centre target: median of the block's subpixel labels; confidence
        // target: share of its integer labels inside [m - h + 1, m + h - 1]
        float v[16];
        int cnt = 0, in = 0;
        for (int yy = 4 * Y; yy < 4 * Y + 4 && yy < H; ++yy)
            for (int xx = 4 * X; xx < 4 * X + 4 && xx < W; ++xx) {
                const size_t p = (size_t)yy * W + xx;
                float a = label_sub[p];
                int k = cnt++;
                for (; k > 0 && v[k - 1] > a; --k) v[k] = v[k - 1];   // insertion sort
                v[k] = a;
                const int d = label_int[p];
                if (d >= mi - h + 1 && d <= mi + h - 1) ++in;
            }
        const float t = (cnt & 1) ? v[cnt / 2] : 0.5f * (v[cnt / 2 - 1] + v[cnt / 2]);
        const float y = (float)in / (float)cnt;
        const float e = c - t, ae = fabsf(e);
        const float huber = ae <= 1.f ? 0.5f * e * e : ae - 0.5f;
        const float bce = fmaxf(z, 0.f) - z * y + log1pf(expf(-fabsf(z)));
        li = y * huber + bce;
        const float invP = 1.f / (float)P;
        const float g0 = 4.f * y * fminf(fmaxf(e, -1.f), 1.f) * invP;
        const float g1 = (1.f / (1.f + expf(-z)) - y) * invP;
        reinterpret_cast<uint4*>(G6)[i] = make_uint4(pack_bf16x2(g0, g1), 0u, 0u, 0u);
    }
    // block sum in a fixed order
    __shared__ float red[kLossThreads];
    red[threadIdx.x] = li;
    __syncthreads();
    for (int s = kLossThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_partial[blockIdx.x] = red[0];
}

__global__ void loss_sum_kernel(const float* __restrict__ loss_partial, int n, int P, float* __restrict__ loss)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) s += loss_partial[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = (float)(red[0] / P);
}

// ---- optimiser and weight packing ----------------------------------------------
__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ grad, int n, float lr, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i];
    const float mi = 0.9f * m[i] + 0.1f * g;
    const float vi = 0.999f * v[i] + 0.001f * g * g;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
}

// Image index e of layer l (forward when dg == 0, data gradient otherwise):
// e = (kc * N + n) * 8 + kk with k = 8 kc + kk.
__global__ void pack_images_kernel(const float* __restrict__ theta, __nv_bfloat16* __restrict__ images)
{
    const int img = blockIdx.y;            // 2 l + dg
    const int l = img >> 1, dg = img & 1;
    if (dg && l == 0) return;
    const int total = dg ? dgrad_image_elems(l) : fwd_image_elems(l);
    const int N = dg ? cin(l) : fwd_n(l);
    const int chp = dg ? cout_pad(l) : cin_pad(l);   // channels of the K dimension (padded)
    __nv_bfloat16* dst = images + (dg ? dgrad_image_offset(l) : fwd_image_offset(l));
    const float* W = theta + param_offset(l);
    const int ci_n = cin(l), co_n = cout(l);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int kk = e & 7, n = (e >> 3) % N, kc = (e >> 3) / N;
        const int k = 8 * kc + kk;
        const int t = k / chp, ch = k % chp;
        float w = 0.f;
        if (t < 9) {
            if (!dg) {
                if (ch < ci_n && n < co_n) w = W[(t * ci_n + ch) * co_n + n];
            } else {
                if (ch < co_n) w = W[(t * ci_n + n) * co_n + ch];
            }
        }
        dst[e] = __float2bfloat16_rn(w);
    }
}

}  // namespace

cudaError_t launch_conv3x3(int cin_ch, int n, const __nv_bfloat16* in, const __nv_bfloat16* image, const float* bias,
                           const __nv_bfloat16* mask, void* out, int nout, int Hq, int Wq, int flip, int mode,
                           int* err, int num_sms, cudaStream_t stream)
{
    if (cin_ch == 8 && n == 32)
        return launch_conv_t<8, 32>(in, image, bias, mask, out, nout, Hq, Wq, flip, mode, err, num_sms, stream);
    if (cin_ch == 32 && n == 32)
        return launch_conv_t<32, 32>(in, image, bias, mask, out, nout, Hq, Wq, flip, mode, err, num_sms, stream);
    if (cin_ch == 32 && n == 16)
        return launch_conv_t<32, 16>(in, image, bias, mask, out, nout, Hq, Wq, flip, mode, err, num_sms, stream);
    return cudaErrorInvalidValue;
}

size_t wgrad_partial_floats(int Hq, int Wq)
{
    const size_t nchunks = ((size_t)Hq * Wq + kWgChunk - 1) / kWgChunk;
    return nchunks * (9 * kWidth * kWidth + kWidth);
}

template <int CIN, int COUT>
cudaError_t launch_wgrad_t(const __nv_bfloat16* X, const __nv_bfloat16* G, int Hq, int Wq, float* partial, int* err,
                           int grid, cudaStream_t stream)
{
    const size_t smem = WgShape<CIN, COUT>::SMEM;
    cudaError_t e = fbs::raise_smem_limit(wgrad_tc_kernel<CIN, COUT>, (int)smem);
    if (e != cudaSuccess) return e;
    fbs::note_launch();
    wgrad_tc_kernel<CIN, COUT><<<grid, kWgThreads, smem, stream>>>(X, G, Hq, Wq, partial, err);
    return cudaGetLastError();
}

cudaError_t launch_wgrad(int l, const __nv_bfloat16* X, const __nv_bfloat16* G, int Hq, int Wq, float* partial,
                         float* grad, int* err, int num_sms, cudaStream_t stream)
{
    const int nchunks = (Hq * Wq + kWgChunk - 1) / kWgChunk;
    // every CTA takes at least one chunk, so every partial is written
    const int grid = nchunks < 2 * num_sms ? nchunks : 2 * num_sms;
    const int cinp = cin_pad(l), coutp = cout_pad(l);
    cudaError_t e;
    if (cinp == 8 && coutp == 32)
        e = launch_wgrad_t<8, 32>(X, G, Hq, Wq, partial, err, grid, stream);
    else if (cinp == 32 && coutp == 32)
        e = launch_wgrad_t<32, 32>(X, G, Hq, Wq, partial, err, grid, stream);
    else if (cinp == 32 && coutp == 8)
        e = launch_wgrad_t<32, 8>(X, G, Hq, Wq, partial, err, grid, stream);
    else
        return cudaErrorInvalidValue;
    if (e != cudaSuccess) return e;
    const int stride = 9 * cinp * coutp + coutp;
    fbs::note_launch();
    wgrad_reduce_kernel<<<(stride + 255) / 256, 256, 0, stream>>>(partial, grid, stride, cinp, coutp, cin(l), cout(l),
                                                                   grad + param_offset(l));
    return cudaGetLastError();
}

int loss_blocks(int P) { return (P + kLossThreads - 1) / kLossThreads; }

cudaError_t launch_loss(const float* out, const int32_t* estar, const int32_t* label_int, const float* label_sub,
                        int H, int W, int D, int half_band, __nv_bfloat16* G6, float* loss_partial, float* loss,
                        cudaStream_t stream)
{
    const int P = ((H + 3) / 4) * ((W + 3) / 4);
    const int nb = loss_blocks(P);
    fbs::note_launch();
    loss_kernel<<<nb, kLossThreads, 0, stream>>>(out, estar, label_int, label_sub, H, W, D, half_band, G6,
                                                  loss_partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    fbs::note_launch();
    loss_sum_kernel<<<1, 256, 0, stream>>>(loss_partial, nb, P, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* theta, float* m, float* v, const float* grad, int n, float lr, float c1, float c2,
                        cudaStream_t stream)
{
    fbs::note_launch();
    adam_kernel<<<(n + 255) / 256, 256, 0, stream>>>(theta, m, v, grad, n, lr, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_pack_images(const float* theta, __nv_bfloat16* images, cudaStream_t stream)
{
    fbs::note_launch();
    pack_images_kernel<<<dim3(16, 2 * kLayers), 256, 0, stream>>>(theta, images);
    return cudaGetLastError();
}

}  // namespace bnet
}  // namespace fbs
