// The learned band form: quarter-resolution features, the band-proposal
// network's forward and training steps, the per-pixel bands and the
// band-restricted path (Eq. (6)-(10) over each pixel's band only).  The
// paper names a reduced search range as the way to avoid filtering the whole
// cost volume (Sec. V); see include/fbs_band.h for the definitions.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "fbs_band.h"
#include "fbs_band_net.cuh"
#include "fbs_context.cuh"

using namespace fbs_detail;

namespace fbs {
namespace {

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// BF16 tensor -> FP32 copy (fbs_band_net_trace)
__global__ void bf16_to_f32_kernel(const __nv_bfloat16* __restrict__ src, float* __restrict__ dst, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = __bfloat162float(src[i]);
}

// ---- features (readings B1-B3) ---------------------------------------------------
// Quarter-resolution intensity of both images: integer sum of the channel
// sums over the 4x4 block, pixels clamped to the image.
__global__ void band_downsample_kernel(const uint8_t* __restrict__ L, const uint8_t* __restrict__ R, int H, int W,
                                       int C, int32_t* __restrict__ gq)
{
    const int Hq = (H + 3) / 4, Wq = (W + 3) / 4;
    const int X = blockIdx.x * blockDim.x + threadIdx.x, Y = blockIdx.y, img = blockIdx.z;
    if (X >= Wq) return;
    const uint8_t* src = img == 0 ? L : R;
    int s = 0;
    for (int j = 0; j < 4; ++j) {
        const int y = min(4 * Y + j, H - 1);
        for (int i = 0; i < 4; ++i) {
            const uint8_t* p = src + ((size_t)y * W + min(4 * X + i, W - 1)) * C;
            s += p[0];
            if (C == 3) s += p[1] + p[2];
        }
    }
    gq[(size_t)img * Hq * Wq + (size_t)Y * Wq + X] = s;
}

// Coarse cost from exact integer sums; the normalisation uses correctly
// rounded FP32 operations in the order of the definition, so every
// evaluation of the same (X, Y, e) gives the same bits.
__device__ __forceinline__ float coarse_from_sums(long long P9, long long Sl, long long Sr, long long Vl,
                                                  long long Vr)
{
    if (Vl == 0 || Vr == 0) return 1.f;
    const long long num = P9 - Sl * Sr;
    const float vv = __fmul_rn(__ll2float_rn(Vl), __ll2float_rn(Vr));
    const float c = __fdiv_rn(__ll2float_rn(num), __fsqrt_rn(vv));
    return __fsub_rn(1.f, c);
}

// Coarse cost volume K [Hq][Wq][Dq] (FP32).  A CTA covers 64 consecutive
// quarter pixels of one row; each thread slides its right block one column
// per e (three new values), and the costs of 32 consecutive e are staged in
// shared memory so that every warp stores 128 contiguous bytes.
constexpr int kCoarseX = 64;
constexpr int kCoarseE = 32;

__global__ void __launch_bounds__(kCoarseX)
band_coarse_cost_kernel(const int32_t* __restrict__ gq, int Hq, int Wq, int Dq, float* __restrict__ K)
{
    __shared__ float tile[kCoarseX][kCoarseE + 1];
    const int X0 = blockIdx.x * kCoarseX, Y = blockIdx.y;
    const int X = X0 + threadIdx.x;
    const bool valid = X < Wq;
    const int32_t* gl = gq;
    const int32_t* gr = gq + (size_t)Hq * Wq;
    const int Xc = valid ? X : Wq - 1;
    int yr[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) yr[j] = clampi(Y - 1 + j, 0, Hq - 1) * Wq;
    long long Sl = 0, Ql = 0;
    int lw[3][3], rw[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            lw[j][i] = gl[yr[j] + clampi(Xc - 1 + i, 0, Wq - 1)];
            Sl += lw[j][i];
            Ql += (long long)lw[j][i] * lw[j][i];
            rw[j][i] = gr[yr[j] + clampi(Xc - 1 + i, 0, Wq - 1)];
        }
    const long long Vl = 9 * Ql - Sl * Sl;
    const int nx = min(kCoarseX, Wq - X0);
    for (int e0 = 0; e0 < Dq; e0 += kCoarseE) {
        const int ne = min(kCoarseE, Dq - e0);
        for (int k = 0; k < ne; ++k) {
            const int e = e0 + k;
            if (e > 0) {
                const int xc = clampi(Xc - e - 1, 0, Wq - 1);
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    rw[j][2] = rw[j][1];
                    rw[j][1] = rw[j][0];
                    rw[j][0] = gr[yr[j] + xc];
                }
            }
            float c = 2.f;
            if (Xc - e >= 0) {
                long long Sr = 0, Qr = 0, P = 0;
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        Sr += rw[j][i];
                        Qr += (long long)rw[j][i] * rw[j][i];
                        P += lw[j][i] * rw[j][i];   // <= 12240^2, exact in int32
                    }
                c = coarse_from_sums(9 * P, Sl, Sr, Vl, 9 * Qr - Sr * Sr);
            }
            tile[threadIdx.x][k] = c;
        }
        __syncthreads();
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int x = warp; x < nx; x += kCoarseX / 32)
            if (lane < ne) K[((size_t)Y * Wq + X0 + x) * Dq + e0 + lane] = tile[x][lane];
        __syncthreads();
    }
}

// Reading B3: row sums over the clipped 5-column window (X' ascending) ...
constexpr int kAggR = 2;

__global__ void band_row_sum_kernel(const float* __restrict__ K, int Hq, int Wq, int Dq, float* __restrict__ Kh)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)Hq * Wq * Dq) return;
    const int e = (int)(i % Dq);
    const size_t q = i / Dq;
    const int X = (int)(q % Wq), Y = (int)(q / Wq);
    float s = 0.f;
    for (int x = max(0, X - kAggR); x <= min(Wq - 1, X + kAggR); ++x) s = __fadd_rn(s, K[((size_t)Y * Wq + x) * Dq + e]);
    Kh[i] = s;
}

// ... then the sum of the row sums (Y' ascending) divided by the tap count.
__global__ void band_col_mean_kernel(const float* __restrict__ Kh, int Hq, int Wq, int Dq, float* __restrict__ Kb)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)Hq * Wq * Dq) return;
    const int e = (int)(i % Dq);
    const size_t q = i / Dq;
    const int X = (int)(q % Wq), Y = (int)(q / Wq);
    const int y0 = max(0, Y - kAggR), y1 = min(Hq - 1, Y + kAggR);
    const int x0 = max(0, X - kAggR), x1 = min(Wq - 1, X + kAggR);
    float s = 0.f;
    for (int y = y0; y <= y1; ++y) s = __fadd_rn(s, Kh[((size_t)y * Wq + X) * Dq + e]);
    Kb[i] = __fdiv_rn(s, (float)((y1 - y0 + 1) * (x1 - x0 + 1)));
}

// One thread per quarter pixel: winner of Kbar (smallest e on ties), the best
// non-adjacent cost and the winner's neighbours give the six features; x0
// receives them as BF16 [P][8] (two zero channels), feat (nullable) as FP32
// [P][6], estar the winner.
__global__ void __launch_bounds__(128)
band_features_kernel(const int32_t* __restrict__ gq, const float* __restrict__ Kb, int H, int W, int C, int D,
                     __nv_bfloat16* __restrict__ x0, float* __restrict__ feat, int32_t* __restrict__ estar)
{
    const int Hq = (H + 3) / 4, Wq = (W + 3) / 4, Dq = (D + 3) / 4;
    const int X = blockIdx.x * blockDim.x + threadIdx.x, Y = blockIdx.y;
    if (X >= Wq) return;
    const size_t i = (size_t)Y * Wq + X;
    const float* k = Kb + i * Dq;
    int best = 0;
    float k1 = k[0];
    for (int e = 1; e < Dq; ++e) {
        const float v = k[e];
        if (v < k1) {
            k1 = v;
            best = e;
        }
    }
    float k2 = 2.f;
    for (int e = 0; e < Dq; ++e)
        if (abs(e - best) >= 2 && k[e] < k2) k2 = k[e];
    const float km = best > 0 ? k[best - 1] : 2.f;
    const float kp = best < Dq - 1 ? k[best + 1] : 2.f;
    float f[6];
    f[0] = __fsub_rn(__fdiv_rn((float)gq[i], (float)(16 * 255 * C)), 0.5f);
    f[1] = __fdiv_rn((float)best, (float)Dq);
    f[2] = k1;
    const float margin = __fsub_rn(k2, k1);
    f[3] = margin < 1.f ? margin : 1.f;
    f[4] = __fsub_rn(km, k1);
    f[5] = __fsub_rn(kp, k1);
    estar[i] = best;
    __nv_bfloat162 h[4];
    h[0] = __floats2bfloat162_rn(f[0], f[1]);
    h[1] = __floats2bfloat162_rn(f[2], f[3]);
    h[2] = __floats2bfloat162_rn(f[4], f[5]);
    h[3] = __floats2bfloat162_rn(0.f, 0.f);
    reinterpret_cast<uint4*>(x0)[i] = *reinterpret_cast<const uint4*>(h);
    if (feat) {
#pragma unroll
        for (int c = 0; c < 6; ++c) feat[i * 6 + c] = f[c];
    }
}

// ---- feature-point proposal (reading B7) -------------------------------------------
// Reliable feature points (margin f3 >= theta_m) of the 5x5 quarter window
// around a pixel's quarter pixel suggest its band: with at least 3 of them and
// a winner spread <= 2 the centre is 2 (max + min) and the confidence 1.
__global__ void band_feature_points_kernel(const float* __restrict__ feat, const int32_t* __restrict__ estar,
                                           int H, int W, float theta_m, float* __restrict__ centre,
                                           float* __restrict__ conf)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W) return;
    const int Hq = (H + 3) / 4, Wq = (W + 3) / 4;
    const int Y = y >> 2, X = x >> 2;
    int n = 0, emin = 1 << 30, emax = -1;
    for (int j = max(0, Y - 2); j <= min(Hq - 1, Y + 2); ++j)
        for (int i = max(0, X - 2); i <= min(Wq - 1, X + 2); ++i) {
            const size_t q = (size_t)j * Wq + i;
            if (!(feat[q * 6 + 3] >= theta_m)) continue;
            ++n;
            emin = min(emin, estar[q]);
            emax = max(emax, estar[q]);
        }
    const size_t p = (size_t)y * W + x;
    const bool ok = n >= 3 && emax - emin <= 2;
    centre[p] = ok ? 2.f * (float)(emax + emin) : 0.f;
    conf[p] = ok ? 1.f : 0.f;
}

// ---- band rule (reading B4) and the per-tile ranges -----------------------------
__device__ __forceinline__ uint32_t band_of(float c, float k, int D, int h, float theta)
{
    if (!(k >= theta) || !isfinite(c)) return (uint32_t)(D - 1) << 16;
    float m = floorf(__fadd_rn(c, 0.5f));
    if (m < 0.f) m = 0.f;
    if (m > (float)(D - 1)) m = (float)(D - 1);
    const int mi = (int)m;
    const int lo = max(mi - h, 0), hi = min(mi + h, D - 1);
    return (uint32_t)lo | ((uint32_t)hi << 16);
}

__global__ void band_limits_kernel(const float* __restrict__ centre, const float* __restrict__ conf, int n, int D,
                                   int h, float theta, int32_t* __restrict__ lo, int32_t* __restrict__ hi)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t b = band_of(centre[i], conf[i], D, h, theta);
    lo[i] = (int32_t)(b & 0xffffu);
    hi[i] = (int32_t)(b >> 16);
}

// One CTA per aggregation tile (one thread per tile pixel).
__global__ void __launch_bounds__(kAggTileX * kAggTileY)
band_tiles_kernel(const float* __restrict__ centre, const float* __restrict__ conf, int H, int W, int D, int h,
                  float theta, uint32_t* __restrict__ band, int2* __restrict__ tile_range)
{
    __shared__ int lo_s, hi_s;
    if (threadIdx.x == 0) {
        lo_s = D;
        hi_s = 0;
    }
    __syncthreads();
    const int x = blockIdx.x * kAggTileX + threadIdx.x % kAggTileX;
    const int y = blockIdx.y * kAggTileY + threadIdx.x / kAggTileX;
    if (x < W && y < H) {
        const size_t p = (size_t)y * W + x;
        const uint32_t b = band_of(centre[p], conf[p], D, h, theta);
        band[p] = b;
        atomicMin(&lo_s, (int)(b & 0xffffu));
        atomicMax(&hi_s, (int)(b >> 16));
    }
    __syncthreads();
    if (threadIdx.x == 0) tile_range[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = make_int2(lo_s & ~3, hi_s + 1);
}

// ---- network head: full-resolution centre and confidence -------------------------
__global__ void band_head_kernel(const float* __restrict__ out, const int32_t* __restrict__ estar, int H, int W,
                                 float* __restrict__ centre, float* __restrict__ conf)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W) return;
    const int Wq = (W + 3) / 4;
    const size_t i = (size_t)(y >> 2) * Wq + (x >> 2);
    const size_t p = (size_t)y * W + x;
    if (centre) centre[p] = __fmul_rn(4.f, __fadd_rn((float)estar[i], out[2 * i]));
    if (conf) conf[p] = 1.f / (1.f + expf(-out[2 * i + 1]));
}

}  // namespace

cudaError_t launch_band_tiles(const float* centre, const float* conf, int H, int W, int D, int half_band,
                              float theta, uint32_t* band, int2* tile_range, cudaStream_t stream)
{
    dim3 grid((W + kAggTileX - 1) / kAggTileX, (H + kAggTileY - 1) / kAggTileY);
    fbs::note_launch();
    band_tiles_kernel<<<grid, kAggTileX * kAggTileY, 0, stream>>>(centre, conf, H, W, D, half_band, theta, band,
                                                                 tile_range);
    return cudaGetLastError();
}

}  // namespace fbs

// ---- state of the network in a context -------------------------------------------
using namespace fbs::bnet;

struct fbs_band_state {
    void* pmem = nullptr;            // parameters, optimiser state, packed images
    float* theta = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    float* grad = nullptr;
    float* loss = nullptr;
    __nv_bfloat16* images = nullptr;
    long long step = 0;
    bool ready = false;
    // shape of the last forward or training call, for fbs_band_net_trace
    int last_H = 0, last_W = 0, last_D = 0;
    bool last_training = false;
};

namespace {

size_t al256(size_t n) { return (n + 255) & ~(size_t)255; }

// Scratch of one quarter-resolution problem, carved from ctx->band_ws.
struct NetScratch {
    int32_t* gq;                 // [2][P]
    float* kq;                   // coarse costs [P][Dq], then their 5x5 means
    float* kh;                   // row sums [P][Dq]
    int32_t* estar;              // [P]
    float* featf;                // [P][6] FP32 features (feature-point proposal)
    __nv_bfloat16* x0;           // [P][8]
    __nv_bfloat16* y[5];         // [P][32]
    float* out;                  // [P][2]
    __nv_bfloat16* g[6];         // gradient w.r.t. the output of layer l: [P][32], g[5] = [P][8]
    float* partial;              // weight-gradient partials
    float* loss_partial;
    float* centre;               // [H][W] (learned entry point)
    float* conf;
    uint32_t* band;              // [H][W]
    int2* tile_range;
};

size_t net_scratch_bytes(int H, int W, int D, bool training, bool full_res)
{
    const size_t Hq = (H + 3) / 4, Wq = (W + 3) / 4, P = Hq * Wq, Dq = (D + 3) / 4;
    size_t n = al256(2 * P * 4) + 2 * al256(P * Dq * 4) + al256(P * 4) + al256(P * 24) + al256(P * 16) + 5 * al256(P * 64) + al256(P * 8);
    if (training)
        n += 5 * al256(P * 64) + al256(P * 16) + al256(wgrad_partial_floats((int)Hq, (int)Wq) * 4) +
             al256((size_t)loss_blocks((int)P) * 4);
    if (full_res) {
        const size_t px = (size_t)H * W;
        const size_t tiles = (size_t)((W + fbs::kAggTileX - 1) / fbs::kAggTileX) * ((H + fbs::kAggTileY - 1) / fbs::kAggTileY);
        n += 3 * al256(px * 4) + al256(tiles * 8);
    }
    return n;
}

NetScratch carve_net(void* base, int H, int W, int D, bool training, bool full_res)
{
    const size_t Hq = (H + 3) / 4, Wq = (W + 3) / 4, P = Hq * Wq, Dq = (D + 3) / 4;
    uint8_t* q = (uint8_t*)base;
    auto take = [&](size_t bytes) {
        void* r = q;
        q += al256(bytes);
        return r;
    };
    NetScratch s{};
    s.gq = (int32_t*)take(2 * P * 4);
    s.kq = (float*)take(P * Dq * 4);
    s.kh = (float*)take(P * Dq * 4);
    s.estar = (int32_t*)take(P * 4);
    s.featf = (float*)take(P * 24);
    s.x0 = (__nv_bfloat16*)take(P * 16);
    for (int l = 0; l < 5; ++l) s.y[l] = (__nv_bfloat16*)take(P * 64);
    s.out = (float*)take(P * 8);
    if (training) {
        for (int l = 0; l < 5; ++l) s.g[l] = (__nv_bfloat16*)take(P * 64);
        s.g[5] = (__nv_bfloat16*)take(P * 16);
        s.partial = (float*)take(wgrad_partial_floats((int)Hq, (int)Wq) * 4);
        s.loss_partial = (float*)take((size_t)loss_blocks((int)P) * 4);
    }
    if (full_res) {
        const size_t px = (size_t)H * W;
        const size_t tiles = (size_t)((W + fbs::kAggTileX - 1) / fbs::kAggTileX) * ((H + fbs::kAggTileY - 1) / fbs::kAggTileY);
        s.centre = (float*)take(px * 4);
        s.conf = (float*)take(px * 4);
        s.band = (uint32_t*)take(px * 4);
        s.tile_range = (int2*)take(tiles * 8);
    }
    return s;
}

fbs_status ensure_state(fbs_ctx* ctx)
{
    if (ctx->band) return FBS_OK;
    fbs_band_state* b = new (std::nothrow) fbs_band_state();
    if (!b) return fail(ctx, FBS_ERR_OOM, "band state");
    const size_t np = al256((size_t)kParams * 4);
    const size_t bytes = 4 * np + 256 + al256((size_t)kImageElems * 2);
    cudaError_t e = cudaMalloc(&b->pmem, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return fail(ctx, FBS_ERR_OOM, "cudaMalloc(%zu) for the band network: %s", bytes, cudaGetErrorString(e));
    }
    uint8_t* q = (uint8_t*)b->pmem;
    b->theta = (float*)q;
    b->m = (float*)(q + np);
    b->v = (float*)(q + 2 * np);
    b->grad = (float*)(q + 3 * np);
    b->loss = (float*)(q + 4 * np);
    b->images = (__nv_bfloat16*)(q + 4 * np + 256);
    ctx->band = b;
    return FBS_OK;
}

fbs_status need_ready(fbs_ctx* ctx)
{
    if (!ctx->band || !ctx->band->ready)
        return fail(ctx, FBS_ERR_INVALID_ARG, "band network has no weights: call fbs_band_net_init or _load first");
    return FBS_OK;
}

// splitmix64 and a Box-Muller normal, for the initial weights
uint64_t splitmix64(uint64_t& s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double uniform01(uint64_t& s) { return ((splitmix64(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

fbs_status upload_params(fbs_ctx* ctx, const float* host, cudaStream_t st)
{
    fbs_band_state* b = ctx->band;
    cudaError_t e = cudaMemcpyAsync(b->theta, host, (size_t)kParams * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->m, 0, (size_t)kParams * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->v, 0, (size_t)kParams * 4, st);
    if (e == cudaSuccess) {
        LaunchScope ls(ctx, FBS_KERNEL_NET, st);
        e = launch_pack_images(b->theta, b->images, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "band network upload");
    b->step = 0;
    b->ready = true;
    return FBS_OK;
}

fbs_status check_pair_shape(fbs_ctx* ctx, const uint8_t* left, const uint8_t* right, int H, int W, int C, int D)
{
    if (!left || !right) return fail(ctx, FBS_ERR_INVALID_ARG, "null image pointer");
    fbs_status s = check_shape(ctx, H, W, C, D);
    if (s != FBS_OK) return s;
    if (ctx->opt.cost != FBS_COST_NCC) return fail(ctx, FBS_ERR_UNSUPPORTED, "the band form uses the NCC cost only");
    return FBS_OK;
}

// Features into the scratch (and optionally the caller's buffers).
fbs_status run_features(fbs_ctx* ctx, const NetScratch& s, const uint8_t* L, const uint8_t* R, int H, int W, int C,
                        int D, float* feat, cudaStream_t st)
{
    const int Hq = (H + 3) / 4, Wq = (W + 3) / 4;
    cudaError_t e;
    {
        LaunchScope ls(ctx, FBS_KERNEL_NET, st);
        fbs::note_launch();
        fbs::band_downsample_kernel<<<dim3((Wq + 127) / 128, Hq, 2), 128, 0, st>>>(L, R, H, W, C, s.gq);
        e = cudaGetLastError();
    }
    const int Dq = (D + 3) / 4;
    const size_t nv = (size_t)Hq * Wq * Dq;
    if (e == cudaSuccess) {
        LaunchScope ls(ctx, FBS_KERNEL_NET, st);
        fbs::note_launch();
        fbs::band_coarse_cost_kernel<<<dim3((Wq + fbs::kCoarseX - 1) / fbs::kCoarseX, Hq), fbs::kCoarseX, 0, st>>>(
            s.gq, Hq, Wq, Dq, s.kq);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        LaunchScope ls(ctx, FBS_KERNEL_NET, st);
        fbs::note_launch();
        fbs::band_row_sum_kernel<<<(unsigned)((nv + 255) / 256), 256, 0, st>>>(s.kq, Hq, Wq, Dq, s.kh);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        LaunchScope ls(ctx, FBS_KERNEL_NET, st);
        fbs::note_launch();
        fbs::band_col_mean_kernel<<<(unsigned)((nv + 255) / 256), 256, 0, st>>>(s.kh, Hq, Wq, Dq, s.kq);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        LaunchScope ls(ctx, FBS_KERNEL_NET, st);
        fbs::note_launch();
        fbs::band_features_kernel<<<dim3((Wq + 127) / 128, Hq), 128, 0, st>>>(s.gq, s.kq, H, W, C, D, s.x0, feat,
                                                                              s.estar);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? FBS_OK : cuda_fail(ctx, e, "band feature launch");
}

// The six convolutions: x0 -> y[0..4] -> out.
fbs_status run_forward(fbs_ctx* ctx, const NetScratch& s, int Hq, int Wq, cudaStream_t st)
{
    fbs_band_state* b = ctx->band;
    const __nv_bfloat16* in = s.x0;
    for (int l = 0; l < kLayers; ++l) {
        const bool last = l == kLayers - 1;
        const float* bias = b->theta + param_offset(l) + 9 * cin(l) * cout(l);
        cudaError_t e;
        {
            LaunchScope ls(ctx, FBS_KERNEL_NET, st);
            e = launch_conv3x3(cin_pad(l), fwd_n(l), in, b->images + fwd_image_offset(l), bias, nullptr,
                               last ? (void*)s.out : (void*)s.y[l], last ? kOut : fwd_n(l), Hq, Wq, 0,
                               last ? kConvLinearF32 : kConvReluBf16, ctx->derr, ctx->num_sms, st);
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "band network convolution launch");
        if (!last) in = s.y[l];
    }
    return FBS_OK;
}

// Loss, backward pass into b->grad.
fbs_status run_backward(fbs_ctx* ctx, const NetScratch& s, int H, int W, int D, const int32_t* label_int,
                        const float* label_sub, int half_band, cudaStream_t st)
{
    fbs_band_state* b = ctx->band;
    const int Hq = (H + 3) / 4, Wq = (W + 3) / 4;
    cudaError_t e;
    {
        LaunchScope ls(ctx, FBS_KERNEL_NET, st);
        e = launch_loss(s.out, s.estar, label_int, label_sub, H, W, D, half_band, s.g[5], s.loss_partial, b->loss, st);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "band loss launch");
    for (int l = kLayers - 1; l >= 0; --l) {
        const __nv_bfloat16* X = l == 0 ? s.x0 : s.y[l - 1];
        {
            LaunchScope ls(ctx, FBS_KERNEL_NET, st);
            e = launch_wgrad(l, X, s.g[l], Hq, Wq, s.partial, b->grad, ctx->derr, ctx->num_sms, st);
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "band weight-gradient launch");
        if (l == 0) break;
        {
            // gradient w.r.t. Y_{l-1} through its ReLU
            LaunchScope ls(ctx, FBS_KERNEL_NET, st);
            e = launch_conv3x3(cout_pad(l), cin(l), s.g[l], b->images + dgrad_image_offset(l), nullptr, s.y[l - 1],
                               s.g[l - 1], cin(l), Hq, Wq, 1, kConvMaskBf16, ctx->derr, ctx->num_sms, st);
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "band data-gradient launch");
    }
    return FBS_OK;
}

fbs_status run_banded(fbs_ctx* ctx, const fbs_pair* p, const float* centre, const float* conf, int h, float theta,
                      const NetScratch& s, cudaStream_t st)
{
    const int H = p->H, W = p->W, D = p->D;
    const int ld = fbs::padded_ld(D);
    const size_t stats = fbs::cost_scratch_bytes(H, W);
    const size_t need = stats + sizeof(float) * (size_t)H * W * ld;
    fbs_status r = ensure(ctx, &ctx->ws, &ctx->ws_bytes, need, "cost volume");
    if (r != FBS_OK) return r;
    const fbs::CostScratch sc = fbs::carve_cost_scratch(ctx->ws, H, W);
    float* cost = (float*)((uint8_t*)ctx->ws + stats);
    cudaError_t e;
    {
        LaunchScope ls(ctx, FBS_KERNEL_NET, st);
        e = fbs::launch_band_tiles(centre, conf, H, W, D, h, theta, s.band, s.tile_range, st);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "band planning launch");
    {
        LaunchScope ls(ctx, FBS_KERNEL_COST, st);
        e = fbs::launch_cost_band(sc, p->left, p->right, H, W, p->C, D, ld, p->radius, s.tile_range, cost, st);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "band cost launch");
    {
        LaunchScope ls(ctx, FBS_KERNEL_AGG_F32, st);
        e = fbs::launch_aggregate_band(cost, ld, p->left, H, W, p->C, D, p->radius, p->sigma_s, p->sigma_r,
                                       s.tile_range, s.band, p->disp_int, p->disp_subpix, st);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "band aggregation launch");
    return FBS_OK;
}

fbs_status check_band_args(fbs_ctx* ctx, const fbs_pair* p, int h, float theta)
{
    if (!p) return fail(ctx, FBS_ERR_INVALID_ARG, "null pair");
    fbs_status s = fbs::check_path_args(ctx, p->left, p->right, p->H, p->W, p->C, p->D, p->radius, p->sigma_s,
                                        p->sigma_r, p->tau, p->disp_int, p->disp_subpix);
    if (s != FBS_OK) return s;
    if (ctx->opt.cost != FBS_COST_NCC) return fail(ctx, FBS_ERR_UNSUPPORTED, "the band form uses the NCC cost only");
    if (h < 1 || h > 512) return fail(ctx, FBS_ERR_INVALID_ARG, "half_band=%d outside 1..512", h);
    if (std::isnan(theta)) return fail(ctx, FBS_ERR_INVALID_ARG, "conf_threshold is NaN");
    return FBS_OK;
}

}  // namespace

namespace fbs {
void band_free(fbs_ctx* ctx)
{
    if (ctx->band) {
        if (ctx->band->pmem) cudaFree(ctx->band->pmem);
        delete ctx->band;
        ctx->band = nullptr;
    }
    if (ctx->band_ws) cudaFree(ctx->band_ws);
    ctx->band_ws = nullptr;
    ctx->band_ws_bytes = 0;
}
}  // namespace fbs

extern "C" {

size_t fbs_band_net_param_count(void) { return (size_t)kParams; }

fbs_status fbs_band_net_init(fbs_ctx* ctx, uint64_t seed)
{
    if (!ctx) return FBS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    fbs_status s = ensure_state(ctx);
    if (s != FBS_OK) return s;
    std::vector<float> h(kParams, 0.f);
    uint64_t st = seed ^ 0x6A09E667F3BCC909ull;
    for (int l = 0; l < kLayers; ++l) {
        const double sd = std::sqrt(2.0 / (9.0 * cin(l))) * (l == kLayers - 1 ? 0.1 : 1.0);
        float* W = h.data() + param_offset(l);
        for (int i = 0; i < 9 * cin(l) * cout(l); ++i) {
            const double u1 = uniform01(st), u2 = uniform01(st);
            W[i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
    }
    return upload_params(ctx, h.data(), ctx->stream);
}

fbs_status fbs_band_net_set_params(fbs_ctx* ctx, const float* params, size_t n)
{
    if (!ctx || !params) return fail(ctx, FBS_ERR_INVALID_ARG, "null context or parameters");
    if (n != (size_t)kParams) return fail(ctx, FBS_ERR_INVALID_ARG, "expected %d parameters, got %zu", kParams, n);
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(params[i])) return fail(ctx, FBS_ERR_INVALID_ARG, "parameter %zu is not finite", i);
    DeviceGuard g(ctx->device);
    fbs_status s = ensure_state(ctx);
    if (s != FBS_OK) return s;
    return upload_params(ctx, params, ctx->stream);
}

fbs_status fbs_band_net_get_params(fbs_ctx* ctx, float* params, size_t n)
{
    if (!ctx || !params) return fail(ctx, FBS_ERR_INVALID_ARG, "null context or parameters");
    if (n != (size_t)kParams) return fail(ctx, FBS_ERR_INVALID_ARG, "expected %d parameters, got %zu", kParams, n);
    fbs_status s = need_ready(ctx);
    if (s != FBS_OK) return s;
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(params, ctx->band->theta, n * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? FBS_OK : cuda_fail(ctx, e, "band parameters read-back");
}

fbs_status fbs_band_net_save(fbs_ctx* ctx, const char* path)
{
    if (!ctx || !path) return fail(ctx, FBS_ERR_INVALID_ARG, "null context or path");
    std::vector<float> h(kParams);
    fbs_status s = fbs_band_net_get_params(ctx, h.data(), h.size());
    if (s != FBS_OK) return s;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(ctx, FBS_ERR_INVALID_ARG, "cannot open %s for writing", path);
    const uint32_t n = (uint32_t)kParams;
    bool ok = std::fwrite("FBSBAND1", 1, 8, f) == 8 && std::fwrite(&n, 4, 1, f) == 1 &&
              std::fwrite(h.data(), 4, h.size(), f) == h.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? FBS_OK : fail(ctx, FBS_ERR_INVALID_ARG, "short write to %s", path);
}

fbs_status fbs_band_net_load(fbs_ctx* ctx, const char* path)
{
    if (!ctx || !path) return fail(ctx, FBS_ERR_INVALID_ARG, "null context or path");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(ctx, FBS_ERR_INVALID_ARG, "cannot open %s", path);
    char tag[8];
    uint32_t n = 0;
    std::vector<float> h(kParams);
    bool ok = std::fread(tag, 1, 8, f) == 8 && std::memcmp(tag, "FBSBAND1", 8) == 0 && std::fread(&n, 4, 1, f) == 1 &&
              n == (uint32_t)kParams && std::fread(h.data(), 4, h.size(), f) == h.size();
    std::fclose(f);
    if (!ok) return fail(ctx, FBS_ERR_INVALID_ARG, "%s is not a band-network file of %d parameters", path, kParams);
    return fbs_band_net_set_params(ctx, h.data(), h.size());
}

fbs_status fbs_band_features(fbs_ctx* ctx, const uint8_t* left, const uint8_t* right, int H, int W, int C, int D,
                             float* feat, int32_t* estar, void* cuda_stream)
{
    if (!ctx) return FBS_ERR_INVALID_ARG;
    fbs_status s = check_pair_shape(ctx, left, right, H, W, C, D);
    if (s != FBS_OK) return s;
    if (!feat && !estar) return fail(ctx, FBS_ERR_INVALID_ARG, "both outputs are NULL");
    DeviceGuard g(ctx->device);
    cudaStream_t st = pick_stream(ctx, cuda_stream);
    s = ensure(ctx, &ctx->band_ws, &ctx->band_ws_bytes, net_scratch_bytes(H, W, D, false, false), "band scratch");
    if (s != FBS_OK) return s;
    const NetScratch sc = carve_net(ctx->band_ws, H, W, D, false, false);
    s = run_features(ctx, sc, left, right, H, W, C, D, feat, st);
    if (s != FBS_OK || !estar) return s;
    const size_t P = (size_t)((H + 3) / 4) * ((W + 3) / 4);
    cudaError_t e = cudaMemcpyAsync(estar, sc.estar, P * 4, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? FBS_OK : cuda_fail(ctx, e, "coarse winner copy");
}

fbs_status fbs_band_net_forward(fbs_ctx* ctx, const uint8_t* left, const uint8_t* right, int H, int W, int C, int D,
                                float* out_q, float* centre, float* conf, void* cuda_stream)
{
    if (!ctx) return FBS_ERR_INVALID_ARG;
    fbs_status s = check_pair_shape(ctx, left, right, H, W, C, D);
    if (s != FBS_OK) return s;
    if (!out_q && !centre && !conf) return fail(ctx, FBS_ERR_INVALID_ARG, "all outputs are NULL");
    if ((s = need_ready(ctx)) != FBS_OK) return s;
    DeviceGuard g(ctx->device);
    cudaStream_t st = pick_stream(ctx, cuda_stream);
    s = ensure(ctx, &ctx->band_ws, &ctx->band_ws_bytes, net_scratch_bytes(H, W, D, false, false), "band scratch");
    if (s != FBS_OK) return s;
    const NetScratch sc = carve_net(ctx->band_ws, H, W, D, false, false);
    const int Hq = (H + 3) / 4, Wq = (W + 3) / 4;
    if ((s = run_features(ctx, sc, left, right, H, W, C, D, nullptr, st)) != FBS_OK) return s;
    if ((s = run_forward(ctx, sc, Hq, Wq, st)) != FBS_OK) return s;
    ctx->band->last_H = H;
    ctx->band->last_W = W;
    ctx->band->last_D = D;
    ctx->band->last_training = false;
    cudaError_t e = cudaSuccess;
    if (centre || conf) {
        LaunchScope ls(ctx, FBS_KERNEL_NET, st);
        fbs::note_launch();
        fbs::band_head_kernel<<<dim3((W + 255) / 256, H), 256, 0, st>>>(sc.out, sc.estar, H, W, centre, conf);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && out_q)
        e = cudaMemcpyAsync(out_q, sc.out, (size_t)Hq * Wq * 8, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? FBS_OK : cuda_fail(ctx, e, "band network head");
}

fbs_status fbs_band_net_train_step(fbs_ctx* ctx, const uint8_t* left, const uint8_t* right, int H, int W, int C,
                                   int D, const int32_t* label_int, const float* label_sub, int half_band, float lr,
                                   float* loss, float* grad, void* cuda_stream)
{
    if (!ctx) return FBS_ERR_INVALID_ARG;
    fbs_status s = check_pair_shape(ctx, left, right, H, W, C, D);
    if (s != FBS_OK) return s;
    if (!label_int || !label_sub) return fail(ctx, FBS_ERR_INVALID_ARG, "null label pointer");
    if (half_band < 1 || half_band > 512) return fail(ctx, FBS_ERR_INVALID_ARG, "half_band=%d outside 1..512", half_band);
    if (!(std::isfinite(lr) && lr >= 0.f)) return fail(ctx, FBS_ERR_INVALID_ARG, "lr must be finite and >= 0");
    if ((s = need_ready(ctx)) != FBS_OK) return s;
    DeviceGuard g(ctx->device);
    cudaStream_t st = pick_stream(ctx, cuda_stream);
    s = ensure(ctx, &ctx->band_ws, &ctx->band_ws_bytes, net_scratch_bytes(H, W, D, true, false), "band scratch");
    if (s != FBS_OK) return s;
    const NetScratch sc = carve_net(ctx->band_ws, H, W, D, true, false);
    const int Hq = (H + 3) / 4, Wq = (W + 3) / 4;
    fbs_band_state* b = ctx->band;
    if ((s = run_features(ctx, sc, left, right, H, W, C, D, nullptr, st)) != FBS_OK) return s;
    if ((s = run_forward(ctx, sc, Hq, Wq, st)) != FBS_OK) return s;
    if ((s = run_backward(ctx, sc, H, W, D, label_int, label_sub, half_band, st)) != FBS_OK) return s;
    b->last_H = H;
    b->last_W = W;
    b->last_D = D;
    b->last_training = true;
    cudaError_t e = cudaSuccess;
    if (grad) e = cudaMemcpyAsync(grad, b->grad, (size_t)kParams * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, b->loss, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && lr > 0.f) {
        b->step += 1;
        const double c1 = 1.0 / (1.0 - std::pow(0.9, (double)b->step));
        const double c2 = 1.0 / (1.0 - std::pow(0.999, (double)b->step));
        {
            LaunchScope ls(ctx, FBS_KERNEL_NET, st);
            e = launch_adam(b->theta, b->m, b->v, b->grad, kParams, lr, (float)c1, (float)c2, st);
        }
        if (e == cudaSuccess) {
            LaunchScope ls(ctx, FBS_KERNEL_NET, st);
            e = launch_pack_images(b->theta, b->images, st);
        }
    }
    if (e == cudaSuccess && (grad || loss)) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? FBS_OK : cuda_fail(ctx, e, "band training step");
}

fbs_status fbs_band_net_trace(fbs_ctx* ctx, float* acts, float* grads, void* cuda_stream)
{
    if (!ctx) return FBS_ERR_INVALID_ARG;
    if (!acts && !grads) return fail(ctx, FBS_ERR_INVALID_ARG, "both outputs are NULL");
    if (!ctx->band || ctx->band->last_H == 0)
        return fail(ctx, FBS_ERR_INVALID_ARG, "no band-network forward or training call to trace");
    fbs_band_state* b = ctx->band;
    if (grads && !b->last_training)
        return fail(ctx, FBS_ERR_INVALID_ARG, "gradients exist only after fbs_band_net_train_step");
    DeviceGuard g(ctx->device);
    cudaStream_t st = pick_stream(ctx, cuda_stream);
    const int H = b->last_H, W = b->last_W, D = b->last_D;
    const NetScratch sc = carve_net(ctx->band_ws, H, W, D, b->last_training, false);
    const size_t P = (size_t)((H + 3) / 4) * ((W + 3) / 4);
    cudaError_t e = cudaSuccess;
    LaunchScope ls(ctx, FBS_KERNEL_OTHER, st);
    auto convert = [&](const __nv_bfloat16* src, float* dst, size_t n) {
        if (e != cudaSuccess) return;
        fbs::note_launch();
        const int blocks = (int)std::min<size_t>((n + 255) / 256, 1024);
        fbs::bf16_to_f32_kernel<<<blocks, 256, 0, st>>>(src, dst, n);
        e = cudaGetLastError();
    };
    if (acts) {
        float* o = acts;
        convert(sc.x0, o, P * 8);
        o += P * 8;
        for (int l = 0; l < 5; ++l, o += P * 32) convert(sc.y[l], o, P * 32);
        if (e == cudaSuccess) e = cudaMemcpyAsync(o, sc.out, P * 8, cudaMemcpyDeviceToDevice, st);
    }
    if (grads) {
        float* o = grads;
        for (int l = 0; l < 5; ++l, o += P * 32) convert(sc.g[l], o, P * 32);
        convert(sc.g[5], o, P * 8);
    }
    return e == cudaSuccess ? FBS_OK : cuda_fail(ctx, e, "band network trace");
}

fbs_status fbs_band_feature_points(fbs_ctx* ctx, const uint8_t* left, const uint8_t* right, int H, int W, int C,
                                  int D, float margin_threshold, float* centre, float* conf, void* cuda_stream)
{
    if (!ctx) return FBS_ERR_INVALID_ARG;
    fbs_status s = check_pair_shape(ctx, left, right, H, W, C, D);
    if (s != FBS_OK) return s;
    if (!centre || !conf) return fail(ctx, FBS_ERR_INVALID_ARG, "null centre or confidence");
    if (std::isnan(margin_threshold)) return fail(ctx, FBS_ERR_INVALID_ARG, "margin_threshold is NaN");
    DeviceGuard g(ctx->device);
    cudaStream_t st = pick_stream(ctx, cuda_stream);
    s = ensure(ctx, &ctx->band_ws, &ctx->band_ws_bytes, net_scratch_bytes(H, W, D, false, false), "band scratch");
    if (s != FBS_OK) return s;
    const NetScratch sc = carve_net(ctx->band_ws, H, W, D, false, false);
    if ((s = run_features(ctx, sc, left, right, H, W, C, D, sc.featf, st)) != FBS_OK) return s;
    LaunchScope ls(ctx, FBS_KERNEL_NET, st);
    fbs::note_launch();
    fbs::band_feature_points_kernel<<<dim3((W + 255) / 256, H), 256, 0, st>>>(sc.featf, sc.estar, H, W,
                                                                           margin_threshold, centre, conf);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FBS_OK : cuda_fail(ctx, e, "feature-point proposal launch");
}

fbs_status fbs_band_limits(fbs_ctx* ctx, const float* centre, const float* conf, int n, int D, int half_band,
                           float conf_threshold, int32_t* lo, int32_t* hi, void* cuda_stream)
{
    if (!ctx) return FBS_ERR_INVALID_ARG;
    if (!centre || !conf || !lo || !hi) return fail(ctx, FBS_ERR_INVALID_ARG, "null pointer");
    if (n < 1 || D < 1 || D > 1024) return fail(ctx, FBS_ERR_INVALID_ARG, "n=%d or D=%d out of range", n, D);
    if (half_band < 1 || half_band > 512) return fail(ctx, FBS_ERR_INVALID_ARG, "half_band=%d outside 1..512", half_band);
    if (std::isnan(conf_threshold)) return fail(ctx, FBS_ERR_INVALID_ARG, "conf_threshold is NaN");
    DeviceGuard g(ctx->device);
    cudaStream_t st = pick_stream(ctx, cuda_stream);
    LaunchScope ls(ctx, FBS_KERNEL_NET, st);
    fbs::note_launch();
    fbs::band_limits_kernel<<<(n + 255) / 256, 256, 0, st>>>(centre, conf, n, D, half_band, conf_threshold, lo, hi);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FBS_OK : cuda_fail(ctx, e, "band limits launch");
}

fbs_status fbs_compute_disparity_banded(fbs_ctx* ctx, const fbs_pair* pair, const float* centre, const float* conf,
                                        int half_band, float conf_threshold, void* cuda_stream)
{
    if (!ctx) return FBS_ERR_INVALID_ARG;
    fbs_status s = check_band_args(ctx, pair, half_band, conf_threshold);
    if (s != FBS_OK) return s;
    if (!centre || !conf) return fail(ctx, FBS_ERR_INVALID_ARG, "null centre or confidence");
    DeviceGuard g(ctx->device);
    cudaStream_t st = pick_stream(ctx, cuda_stream);
    s = ensure(ctx, &ctx->band_ws, &ctx->band_ws_bytes, net_scratch_bytes(pair->H, pair->W, pair->D, false, true),
               "band scratch");
    if (s != FBS_OK) return s;
    const NetScratch sc = carve_net(ctx->band_ws, pair->H, pair->W, pair->D, false, true);
    return run_banded(ctx, pair, centre, conf, half_band, conf_threshold, sc, st);
}

fbs_status fbs_compute_disparity_learned(fbs_ctx* ctx, const fbs_pair* pair, int half_band, float conf_threshold,
                                         void* cuda_stream)
{
    if (!ctx) return FBS_ERR_INVALID_ARG;
    fbs_status s = check_band_args(ctx, pair, half_band, conf_threshold);
    if (s != FBS_OK) return s;
    if ((s = need_ready(ctx)) != FBS_OK) return s;
    DeviceGuard g(ctx->device);
    cudaStream_t st = pick_stream(ctx, cuda_stream);
    const int H = pair->H, W = pair->W;
    s = ensure(ctx, &ctx->band_ws, &ctx->band_ws_bytes, net_scratch_bytes(H, W, pair->D, false, true), "band scratch");
    if (s != FBS_OK) return s;
    const NetScratch sc = carve_net(ctx->band_ws, H, W, pair->D, false, true);
    const int Hq = (H + 3) / 4, Wq = (W + 3) / 4;
    if ((s = run_features(ctx, sc, pair->left, pair->right, H, W, pair->C, pair->D, nullptr, st)) != FBS_OK) return s;
    if ((s = run_forward(ctx, sc, Hq, Wq, st)) != FBS_OK) return s;
    {
        LaunchScope ls(ctx, FBS_KERNEL_NET, st);
        fbs::note_launch();
        fbs::band_head_kernel<<<dim3((W + 255) / 256, H), 256, 0, st>>>(sc.out, sc.estar, H, W, sc.centre, sc.conf);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "band head launch");
    }
    return run_banded(ctx, pair, sc.centre, sc.conf, half_band, conf_threshold, sc, st);
}

}  // extern "C"
