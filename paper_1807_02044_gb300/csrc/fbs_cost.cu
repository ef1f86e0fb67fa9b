// Step 1 of fast bilateral stereo: the matching-cost volume.
//
// NCC (Sec. II-A, Eq. (1)-(3), varrho = 1): with the intensity g taken as the
// channel sum, n = 9 and the block sums S = sum g, Q = sum g^2 and
// P = sum g_l g_r, Eq. (1) multiplied through by n^2 reads
//     c = (n P - S_l S_r) / sqrt((n Q_l - S_l^2) (n Q_r - S_r^2)).
// Every sum and both numerator terms are exact in int32 (g <= 765), so only the
// final normalisation is rounded.  As the paper pre-computes mu and sigma and
// keeps only the dot product per (p, d) (Sec. II-A, Sec. III), each CTA first
// computes the block statistics of its row segment in shared memory; the
// per-(p, d) work is the 9-term dot product.  Stored cost: C = 1 - c.
// Boundary rules: blocks clamp to the image; u - d < 0 gives the maximum cost;
// a block of zero variance gives c = 0.
//
// TAD (not in the paper): C = min(mean_c |I_l(u,v) - I_r(u-d,v)|, tau).
//
// The kernel is bound by the HBM write of the volume (4 bytes per (p, d));
// consecutive lanes write consecutive d of one pixel, so every warp store is
// one fully used 128-byte line.
#include "fbs_internal.cuh"

namespace fbs {
namespace {

constexpr int kCostXS = 64;        // pixels per CTA along x
constexpr int kCostThreads = 256;  // 8 warps

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ int grey_at(const uint8_t* __restrict__ img, int W, int C, int x, int y)
{
    const uint8_t* p = img + ((size_t)y * W + x) * C;
    int s = p[0];
    if (C == 3) s += p[1] + p[2];
    return s;
}

__global__ void __launch_bounds__(kCostThreads)
cost_build_kernel(const uint8_t* __restrict__ L, const uint8_t* __restrict__ R, int H, int W,
                  int C, int D, int ld, int mode, float tau, float* __restrict__ cost)
{
    extern __shared__ int smem_i[];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * kCostXS;
    const int y = blockIdx.y;
    const int nxs = min(kCostXS, W - x0);
    // left virtual columns x0-1 .. x0+nxs, right virtual columns x0-D .. x0+nxs
    const int nl = nxs + 2;
    const int nr = nxs + D + 1;
    int* gl = smem_i;                       // [3][nl]
    int* gr = gl + 3 * nl;                  // [3][nr]
    int* Sl = gr + 3 * nr;                  // [nxs]    left block sums at x0+i
    float* rl = (float*)(Sl + nxs);         // [nxs]    1/sqrt(V_l), 0 if flat
    int* Sr = (int*)(rl + nxs);             // [nr-2]   right block sums, centre index 1..nr-2
    float* rr = (float*)(Sr + (nr - 2));    // [nr-2]

    if (mode == 0) {
        for (int i = tid; i < 3 * nl; i += kCostThreads) {
            int j = i / nl, c = i - j * nl;
            gl[i] = grey_at(L, W, C, clampi(x0 - 1 + c, 0, W - 1), clampi(y - 1 + j, 0, H - 1));
        }
        for (int i = tid; i < 3 * nr; i += kCostThreads) {
            int j = i / nr, c = i - j * nr;
            gr[i] = grey_at(R, W, C, clampi(x0 - D + c, 0, W - 1), clampi(y - 1 + j, 0, H - 1));
        }
        __syncthreads();
        for (int i = tid; i < nxs; i += kCostThreads) {
            int s = 0, q = 0;
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    int g = gl[j * nl + i + k];
                    s += g;
                    q += g * g;
                }
            int v = 9 * q - s * s;
            Sl[i] = s;
            rl[i] = v > 0 ? rsqrtf((float)v) : 0.f;
        }
        for (int i = tid; i < nr - 2; i += kCostThreads) {
            int s = 0, q = 0;
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    int g = gr[j * nr + i + k];
                    s += g;
                    q += g * g;
                }
            int v = 9 * q - s * s;
            Sr[i] = s;
            rr[i] = v > 0 ? rsqrtf((float)v) : 0.f;
        }
        __syncthreads();
    }

    const int warp = tid >> 5, lane = tid & 31;
    const float inv_c = 1.f / (float)C;
    for (int i = warp; i < nxs; i += kCostThreads / 32) {
        const int x = x0 + i;
        float* out = cost + ((size_t)y * W + x) * ld;
        for (int d = lane; d < ld; d += 32) {
            float cst;
            if (d >= D) {
                cst = 0.f;
            } else if (x - d < 0) {
                cst = mode == 0 ? 2.f : tau;
            } else if (mode == 0) {
                const int rc = i + D - d;   // index of the right block centre (virtual column x-d)
                int P = 0;
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int k = 0; k < 3; ++k) P += gl[j * nl + i + k] * gr[j * nr + rc - 1 + k];
                const int num = 9 * P - Sl[i] * Sr[rc - 1];
                const float c = (float)num * (rl[i] * rr[rc - 1]);
                cst = 1.f - c;
            } else {
                const uint8_t* pl = L + ((size_t)y * W + x) * C;
                const uint8_t* pr = R + ((size_t)y * W + (x - d)) * C;
                int s = 0;
                for (int c = 0; c < C; ++c) s += abs((int)pl[c] - (int)pr[c]);
                cst = fminf((float)s * inv_c, tau);
            }
            out[d] = cst;
        }
    }
}

}  // namespace

cudaError_t launch_cost_build(const uint8_t* left, const uint8_t* right, int H, int W, int C,
                              int D, int ld, int mode, float tau, float* cost, cudaStream_t stream)
{
    const int nxs = kCostXS;
    const int nl = nxs + 2, nr = nxs + D + 1;
    const size_t smem = sizeof(int) * (size_t)(3 * nl + 3 * nr + 2 * nxs + 2 * (nr - 2));
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(cost_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((W + kCostXS - 1) / kCostXS, H);
    cost_build_kernel<<<grid, kCostThreads, smem, stream>>>(left, right, H, W, C, D, ld, mode, tau, cost);
    return cudaGetLastError();
}

}  // namespace fbs
