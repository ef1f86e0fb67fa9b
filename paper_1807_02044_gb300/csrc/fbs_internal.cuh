// Internal declarations shared by the translation units of libfbs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fbs.h"

namespace fbs {

// Kernels launched by the calling host thread (every launch site notes itself;
// a context's per-kind counters add the difference around each launch scope).
extern thread_local long long tl_kernel_launches;
inline void note_launch() { ++tl_kernel_launches; }
inline long long launch_count() { return tl_kernel_launches; }

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) costs a driver call per
// launch; this raises a kernel's limit on the current device only when a
// launch needs more than has been set there before (thread-safe).
cudaError_t raise_smem_limit(const void* kernel, size_t bytes);
template <typename K>
inline cudaError_t raise_smem_limit(K* kernel, size_t bytes)
{
    return raise_smem_limit((const void*)kernel, bytes);
}

// Cost volume rows are padded to a multiple of 4 floats so that one pixel's
// disparity vector starts on a 16-byte boundary (vector loads, TMA, cp.async).
inline int padded_ld(int D) { return (D + 3) & ~3; }

// ---- step 1: matching cost, Eq. (1)-(3) or TAD -------------------------------
// Per-pixel statistics of both images (grey value, 3x3 block sum, 1/sqrt of
// the block variance times n^2), computed by a pre-pass and read by the FP32
// layout's cost kernels (the 16-bit x-blocked cost kernel computes them in
// shared memory and uses only rgbx).  Both images: 2*H*W entries each.
struct CostScratch {
    int16_t* g;
    int* s;
    float* rv;
    uint2* rgbx;      // optional: left image as (R | G << 8 | B << 16, R^2 + G^2 + B^2), pitch rgbx_pitch(W)
};
size_t cost_scratch_bytes(int H, int W);
CostScratch carve_cost_scratch(void* base, int H, int W);
// Size and carving of the optional packed guide plane that follows the statistics.
size_t rgbx_bytes(int H, int W);
__host__ __device__ inline int rgbx_pitch(int W) { return (W + 1) & ~1; }

// cost[(y*W + x)*ld + d] for d < D; entries D <= d < ld are written as 0.
cudaError_t launch_cost_build(const CostScratch& sc, const uint8_t* left, const uint8_t* right, int H, int W,
                              int C, int D, int ld, int mode, float tau, float* cost, cudaStream_t stream);

// Both views (Sec. II-A, Sec. III): cost as launch_cost_build, and cost_r
// [H][W][ld] the right volume, cost_r(x, y, d) = cost(x + d, y, d), the maximum
// cost where x + d >= W.
cudaError_t launch_cost_build_lr(const CostScratch& sc, const uint8_t* left, const uint8_t* right, int H, int W,
                                 int C, int D, int ld, int mode, float tau, float* cost, float* cost_r,
                                 cudaStream_t stream);

// 16-bit x-blocked volume cost[((y*ceil(W/8) + x/8)*Dp + d)*8 + x%8] with
// Dp = tc_block_rows(D) = round_up(D,16) + 16 rows per block: d < D the cost,
// D <= d < round_up(D,16) zero, row round_up(D,16) all ones and the 15 rows
// after it zero -- the ones row lets the tensor-core product also form the sum
// of the weights.  Columns x >= W of the last block are 0.  bf16 selects
// __nv_bfloat16, otherwise __half.  One kernel, which also writes the left
// image's packed guide to sc.rgbx (required; the statistics planes of sc are
// not used).  D <= 256 (Dp <= 272).
__host__ __device__ inline int tc_block_rows(int D) { return (D + 15) / 16 * 16 + 16; }
inline size_t xblock16_bytes(int H, int W, int D) { return (size_t)H * ((W + 7) / 8) * tc_block_rows(D) * 8 * 2; }
cudaError_t launch_cost_build_xblock16(const CostScratch& sc, const uint8_t* left, const uint8_t* right, int H,
                                       int W, int C, int D, int mode, float tau, bool bf16, void* cost,
                                       cudaStream_t stream);

// ---- steps 2-4 in FP32: Eq. (6)-(8), WTA, Eq. (10) ----------------------------
// Pixel tile of the FP32 aggregation (also the unit of the band form's ranges).
constexpr int kAggTileX = 32;
constexpr int kAggTileY = 4;
// agg_out (nullable) is written with row pitch D (caller layout [H][W][D]).
cudaError_t launch_aggregate_f32(const float* cost, int ld, const uint8_t* guide, int H, int W,
                                 int C, int D, int radius, float sigma_s, float sigma_r,
                                 float* agg_out, int32_t* disp_int, float* disp_sub,
                                 cudaStream_t stream);

// ---- steps 2-4 on the tensor cores (BF16 / FP16 operands, FP32 accumulate) ---
// cost: 16-bit x-blocked volume (see launch_cost_build_xblock16), 16-byte
// aligned.  err: device int set to nonzero if a bounded wait inside the kernel
// gave up.
int tc_supported(int D, int radius);
// max_rows (0 = the kernel's own maximum) caps the window rows per pipeline
// stage; wait_cycles (0 = about 2 s) limits each pipeline wait of the kernel.
cudaError_t launch_aggregate_tc(const void* cost, const uint2* rgbx, int H, int W, int C, int D,
                                int radius, float sigma_s, float sigma_r, bool bf16, float* agg_out,
                                int32_t* disp_int, float* disp_sub, int* err, int num_sms, cudaStream_t stream,
                                int max_rows = 0, long long wait_cycles = 0);
// Persistent tensor-core aggregation over a batch.  The members are grouped
// by the producers' column-pair variant (a function of the radius); one
// persistent launch per group walks the tiles of all its members (largest
// tiles first, CTA b takes work items b, b + grid, ...), each member with its
// own tensor maps, size and D, read from a device table.  tc_batch_prepare
// fills the table (host memory of tc_batch_table_bytes(n) bytes, to be copied
// to a device buffer of that size that stays allocated while launches use it)
// and the launch description; the per-pixel results equal
// launch_aggregate_tc's bit for bit.
struct TcBatchMember {
    const void* cost;      // 16-bit x-blocked volume written by launch_cost_build_xblock16
    const uint2* rgbx;     // its packed guide
    int H, W, C, D, radius;
    float sigma_s, sigma_r;
    int32_t* disp_int;
    float* disp_sub;
};
struct TcBatchGroup {
    int variant, first, npairs, nitems;    // members first .. first + npairs - 1 of the table
    int R, S, nacc, kw_max, nh_max;
    uint32_t a_stage, b_stage, acc_stride, tmem_cols;
    size_t smem;
};
struct TcBatchLaunch {
    int ngroups;
    TcBatchGroup group[18];
};
size_t tc_batch_table_bytes(int n);
cudaError_t tc_batch_prepare(int n, const TcBatchMember* members, bool bf16, void* host_table, TcBatchLaunch* out);
// Launches every group in order on `stream` (one kernel each).
cudaError_t launch_aggregate_tc_batch(const void* dev_table, const TcBatchLaunch& launch, bool bf16, int* err,
                                      int num_sms, long long wait_cycles, cudaStream_t stream);
// Packed guide plane of an image: (RGBX, squared norm) per pixel, pitch rgbx_pitch(W); the
// tensor-core path loads its guide tiles from it.
cudaError_t launch_pack_rgbx(const uint8_t* img, int H, int W, int C, uint2* rgbx, cudaStream_t stream);
// FP32 [H][W][D] -> 16-bit x-blocked volume (rounded to nearest).
cudaError_t launch_hwd_to_xblock16(const float* in, int H, int W, int D, bool bf16, void* out, cudaStream_t stream);
// Rows D .. Dp-1 of every block of the x-blocked volume (zeros and the ones row).
cudaError_t launch_xblock16_pad_rows(int H, int W, int D, bool bf16, void* out, cudaStream_t stream);

// ---- band form: per-pixel disparity bands ---------------------------------------
// band[p] = lo | (hi << 16): pixel p searches [lo, hi].  tile_range[t] =
// (d_begin, d_end) of aggregation tile t (kAggTileX x kAggTileY pixels,
// row-major tiles): d_begin = min lo rounded down to a multiple of 4, d_end =
// max hi + 1.  The statistics pre-pass runs inside launch_cost_band.
cudaError_t launch_band_tiles(const float* centre, const float* conf, int H, int W, int D, int half_band,
                              float theta, uint32_t* band, int2* tile_range, cudaStream_t stream);
cudaError_t launch_cost_band(const CostScratch& sc, const uint8_t* left, const uint8_t* right, int H, int W,
                             int C, int D, int ld, int radius, const int2* tile_range, float* cost,
                             cudaStream_t stream);
cudaError_t launch_aggregate_band(const float* cost, int ld, const uint8_t* guide, int H, int W, int C, int D,
                                  int radius, float sigma_s, float sigma_r, const int2* tile_range,
                                  const uint32_t* band, int32_t* disp_int, float* disp_sub, cudaStream_t stream);

// ---- batched form: one persistent launch per stage over many pairs ------------
// Device-side description of one pair of a batch.  *_off is the index of the
// pair's first work item in each batched kernel (items of a pair contiguous,
// pairs in batch order, offsets ascending).
struct BatchPair {
    const uint8_t* left;
    const uint8_t* right;
    int H, W, C, D, radius, ld, mode;
    float neg_ks, neg_kr, tau;
    CostScratch sc;
    float* cost;
    int32_t* disp_int;
    float* disp_sub;
    int stat_off, cost_off, agg_off;
};
#ifdef __CUDACC__
__device__ __forceinline__ int find_pair(const BatchPair* pairs, int n, int item, int BatchPair::*off)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pairs[mid].*off <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}
#endif
// work items per pair
int stats_items(int H, int W);
int cost_items(int H, int W);
int agg_f32_tiles(int H, int W);
size_t cost_kernel_smem();
cudaError_t prepare_cost_batched();
cudaError_t launch_stats_batched(const BatchPair* pairs, int npairs, int nitems, int* counter, int grid,
                                 cudaStream_t stream);
cudaError_t launch_cost_batched(const BatchPair* pairs, int npairs, int nitems, int* counter, int grid,
                                cudaStream_t stream);
cudaError_t prepare_aggregate_f32_batched(int max_radius, size_t* smem_out);
cudaError_t launch_aggregate_f32_batched(const BatchPair* pairs, int npairs, int nitems, int* counter, int grid,
                                         size_t smem, cudaStream_t stream);

// ---- context helpers for entry points defined outside fbs_api.cu -------------
// Host-side checks of fbs_compute_disparity's arguments (sets the message).
fbs_status check_path_args(fbs_ctx* ctx, const uint8_t* left, const uint8_t* right, int H, int W, int C,
                           int D, int radius, float sigma_s, float sigma_r, float tau,
                           const int32_t* disp_int, const float* disp_subpix);
// Release the band form's state (called by fbs_destroy).
void band_free(fbs_ctx* ctx);
// The single-view tensor-core path of fbs_compute_disparity (context scratch
// ctx->ws; arguments already checked).
fbs_status run_path_tc(fbs_ctx* ctx, const uint8_t* left, const uint8_t* right, int H, int W, int C, int D,
                       int radius, float sigma_s, float sigma_r, float tau, int32_t* disp_int, float* disp_subpix,
                       cudaStream_t st);

}  // namespace fbs
