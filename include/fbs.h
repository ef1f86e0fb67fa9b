/*
 * fbs.h -- C ABI of libfbs, fast bilateral stereo (FBS) on one GB300 GPU.
 *
 * The method ("Real-Time Subpixel Fast Bilateral Stereo", Sec. II):
 *   1. matching cost:  normalised cross-correlation of 3x3 blocks, Eq. (1)-(3),
 *                      stored as C = 1 - c in [0, 2];
 *   2. aggregation:    C_agg(p, d) = sum_q w(p,q) C(q,d) / sum_q w(p,q) over the
 *                      (2 radius + 1)^2 window, w = omega_d * omega_r, Eq. (6)-(8);
 *   3. optimisation:   winner-take-all over d, Sec. II-C / III;
 *   4. refinement:     parabola through C_agg(d*-1), C_agg(d*), C_agg(d*+1), Eq. (10).
 *
 * Conventions shared by every entry point:
 *   - Every call returns an fbs_status and never aborts the process.  After a
 *     non-OK status, fbs_last_error() gives a one-line message.
 *   - Images are uint8, row-major HWC (pitch W*C bytes), C = 1 or 3, in DEVICE
 *     memory owned by the caller unless the entry point says "host".
 *   - Cost and aggregated volumes are float32, layout [H][W][D] (D innermost).
 *   - Disparity maps are H*W, int32 (integer winner) and float32 (subpixel).
 *   - Calls are asynchronous on the given CUDA stream (a cudaStream_t passed
 *     as void*; NULL selects the context's own stream).  Errors raised by
 *     kernels surface at the next call or at fbs_sync().
 *   - Arguments are validated on the host before any launch; a violation
 *     returns FBS_ERR_INVALID_ARG and launches nothing.
 *   - Limits: 1 <= H, W <= 16384; C in {1, 3}; 1 <= D <= 1024;
 *     0 <= radius <= 31; sigma_s > 0; sigma_r > 0; tau >= 0 (TAD mode).
 *   - A context is bound to one device and is not thread-safe: use one per
 *     host thread.
 */
#ifndef FBS_H
#define FBS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fbs_ctx fbs_ctx;

typedef enum {
    FBS_OK = 0,
    FBS_ERR_INVALID_ARG = 1,   /* bad pointer, size or parameter */
    FBS_ERR_OOM = 2,           /* device allocation failed or workspace cap reached */
    FBS_ERR_CUDA = 3,          /* a CUDA call or kernel failed; see fbs_last_error */
    FBS_ERR_TIMEOUT = 4,       /* a bounded device-side wait gave up */
    FBS_ERR_UNSUPPORTED = 5    /* valid request outside a form's limits (e.g. D > 256 on the tensor cores) */
} fbs_status;

/* Matching cost.  NCC is the paper's, Eq. (1)-(3) with varrho = 1.  TAD is a
 * truncated mean absolute difference min(mean_c |I_l - I_r|, tau), not in the
 * paper, offered for comparison. */
typedef enum { FBS_COST_NCC = 0, FBS_COST_TAD = 1 } fbs_cost_mode;

/* Arithmetic of the aggregation, Eq. (6).  F32: FP32 FMA.  BF16 / F16: cost
 * and weight tiles rounded to 16 bits, products on the tensor cores with FP32
 * accumulation; normalisation, WTA and Eq. (10) stay FP32. */
typedef enum { FBS_PREC_F32 = 0, FBS_PREC_BF16 = 1, FBS_PREC_F16 = 2 } fbs_precision;

typedef struct {
    int cost;                   /* fbs_cost_mode */
    int prec;                   /* fbs_precision */
    int fused;                  /* reserved, 0 */
    size_t workspace_cap;       /* bytes of scratch the context may hold; 0 = unlimited */
    const char *autotune_cache_path; /* batched form: file of "shape plan" lines the
                                        autotuner appends to and reads back; may be NULL */
} fbs_options;

/* Fill *opt with the defaults: NCC, F32, unfused, no cap, no autotune cache file. */
void fbs_default_options(fbs_options *opt);

/* Create a context on CUDA device `device`.  opt may be NULL (defaults).
 * The context owns its stream and scratch memory; *out receives it. */
fbs_status fbs_create(fbs_ctx **out, const fbs_options *opt, int device);

/* Release everything the context owns.  NULL-safe.  Synchronises its stream. */
fbs_status fbs_destroy(fbs_ctx *ctx);

/* Replace the options of an existing context (cost mode, precision, cap). */
fbs_status fbs_set_options(fbs_ctx *ctx, const fbs_options *opt);

/* Block until all work issued through ctx (on any stream) has finished and
 * report any kernel error. */
fbs_status fbs_sync(fbs_ctx *ctx);

/* Failure detection (not a step of the method).  Every wait of the
 * tensor-core aggregation on another part of the same kernel (its pipeline of
 * weight producers, copies, MMAs and epilogue) is bounded: after `seconds` of
 * SM clock time the kernel stops issuing work, lets its own copies and MMAs
 * land (a fixed ~2 s bound), frees its tensor memory and records an error
 * that the next fbs_sync returns as FBS_ERR_TIMEOUT; the outputs of that call
 * are invalid and the context stays usable.  0 <= seconds <= 60, 0 = the
 * default (about 2 s).  Applies to kernels launched after the call (batch
 * graphs built earlier keep the limit they were built with). */
fbs_status fbs_set_wait_limit(fbs_ctx *ctx, double seconds);

/* Failure injection (a test hook; not a step of the method): the next
 * `count` steps of fbs_compute_disparity or fbs_compute_disparity_host (and
 * of fbs_compute_disparity_lr in BF16 / FP16 contexts) on ctx launch nothing
 * and fail as if their first
 * kernel launch had returned `cuda_error` (a cudaError_t value): FBS_ERR_OOM
 * for cudaErrorMemoryAllocation, FBS_ERR_CUDA otherwise, with the error's
 * text in fbs_last_error.  Lets a caller exercise its error handling without a
 * device fault; the context stays usable.  count 0 disarms; count < 0, or a
 * zero error with count > 0, is FBS_ERR_INVALID_ARG. */
fbs_status fbs_debug_fail_launches(fbs_ctx *ctx, int cuda_error, int count);

/* Message for the last non-OK status of this context ("" if none). */
const char *fbs_last_error(const fbs_ctx *ctx);

/*
 * The whole path (Sec. II-A..II-D; implementation Sec. III): cost volume of
 * the left view, bilateral aggregation guided by the left image, WTA and
 * Eq. (10).  left, right: device images.  disp_int, disp_subpix: device
 * outputs of H*W elements; either may be NULL but not both.  sigma_s is
 * gamma_d of Eq. (7), sigma_r is gamma_r of Eq. (8); tau is used only by the
 * TAD cost mode.  Scratch held by ctx: FP32 -- the block statistics and one
 * cost volume (H*W*round_up(D,4)*4 bytes); BF16 / F16 -- one 16-bit x-blocked
 * cost volume (H*ceil(W/8)*8*Dp*2 bytes, Dp as for the batched form) and the
 * packed guide.  The 16-bit forms need D <= 256 and radius <= 24
 * (FBS_ERR_UNSUPPORTED otherwise).  Two kernels per call in the 16-bit forms
 * (cost build, tensor-core aggregation launched programmatically so its
 * set-up overlaps the end of the cost build), three in FP32.
 */
fbs_status fbs_compute_disparity(fbs_ctx *ctx, const uint8_t *left, const uint8_t *right,
                                 int H, int W, int C, int D, int radius,
                                 float sigma_s, float sigma_r, float tau,
                                 int32_t *disp_int, float *disp_subpix, void *cuda_stream);

/*
 * Same as fbs_compute_disparity with HOST buffers: left/right are read from
 * host memory, results are written to host memory, and the call returns after
 * the results have arrived.  FP32 contexts, or pageable buffers: the images
 * are copied to device staging and the maps back, on the context's stream.
 * BF16 / FP16 contexts with page-locked buffers the GPU can address (all four,
 * or the ones given): no staging copies -- the cost kernel reads the images
 * from host memory and the aggregation writes the maps there directly.
 */
fbs_status fbs_compute_disparity_host(fbs_ctx *ctx, const uint8_t *left, const uint8_t *right,
                                      int H, int W, int C, int D, int radius,
                                      float sigma_s, float sigma_r, float tau,
                                      int32_t *disp_int, float *disp_subpix);

/*
 * Both views and the left-right consistency (LRC) check (Sec. II-A, Sec. III,
 * Eq. (9)).  The right map at (u, v) matches R(u) against L(u + d); where
 * u + d >= W the cost is the maximum.  Each view is aggregated with its own
 * image as guide (Eq. (6)-(8)), WTA and Eq. (10) give both maps.
 *   disp_int / disp_subpix: the LEFT map (either may be NULL, not both); with
 *     lrc != 0 every left pixel whose disparity d fails Eq. (9) -- u - d < 0 or
 *     the right disparity at (u - d, v) differs from d -- is set to -1 in both.
 *   disp_int_right / disp_subpix_right (each nullable): the right map.
 * FP32 context: each matching cost is computed once and stored in the left
 * volume at (u, v, d) and in the right volume at (u - d, v, d); scratch: two
 * cost volumes (2 * H*W*round_up(D,4)*4 bytes) and two integer maps.
 * BF16 / FP16 context: the tensor-core path of fbs_compute_disparity for the
 * left view, and for the right view the same path on the horizontally
 * mirrored pair with the images swapped (its left view is the mirrored right
 * view), mirrored back; the left map is bit-identical to
 * fbs_compute_disparity's.  D <= 256 and radius <= 24 (FBS_ERR_UNSUPPORTED
 * otherwise); scratch: one 16-bit volume at a time plus two mirrored images
 * and four maps.
 */
fbs_status fbs_compute_disparity_lr(fbs_ctx *ctx, const uint8_t *left, const uint8_t *right,
                                    int H, int W, int C, int D, int radius,
                                    float sigma_s, float sigma_r, float tau,
                                    int32_t *disp_int, float *disp_subpix,
                                    int32_t *disp_int_right, float *disp_subpix_right, int lrc,
                                    void *cuda_stream);

/*
 * Step 1 alone, Eq. (1)-(3) (or TAD): writes cost_out[H][W][D] (device,
 * float32, caller-owned).  For u - d < 0 the cost is the maximum (2 for NCC,
 * tau for TAD); a zero-variance block gives c = 0.
 */
fbs_status fbs_cost_volume(fbs_ctx *ctx, const uint8_t *left, const uint8_t *right,
                           int H, int W, int C, int D, float tau, float *cost_out,
                           void *cuda_stream);

/*
 * Steps 2-4 on a given cost volume, Eq. (6)-(8) and Eq. (10): cost[H][W][D]
 * (device float32), guide = the left image (device uint8 HWC).  agg_out
 * (nullable) receives the aggregated volume [H][W][D]; disp_int / disp_subpix
 * as above (all three may not be NULL together).  The cost values are taken
 * as given, so a test can feed any volume (e.g. an exact quadratic in d).
 */
fbs_status fbs_aggregate(fbs_ctx *ctx, const float *cost, const uint8_t *guide,
                         int H, int W, int C, int D, int radius,
                         float sigma_s, float sigma_r,
                         float *agg_out, int32_t *disp_int, float *disp_subpix,
                         void *cuda_stream);

/*
 * Batched form (not a step of the method; a serving form of Sec. II-III):
 * one stereo pair of a batch.  Pointers are device memory owned by the
 * caller; parameters as for fbs_compute_disparity.
 */
typedef struct {
    const uint8_t *left, *right;
    int H, W, C, D, radius;
    float sigma_s, sigma_r, tau;
    int32_t *disp_int;          /* may be NULL */
    float *disp_subpix;         /* may be NULL (not both) */
} fbs_pair;

/*
 * fbs_compute_disparity for n pairs of uneven size, disparity count and
 * radius (1 <= n <= 4096; pairs is a host array), replayed as one CUDA graph
 * per batch shape; results are bit-identical to fbs_compute_disparity in the
 * context's precision.
 *   FP32: either each stage (block statistics, cost volumes, aggregation
 *   with WTA and Eq. (10)) is one persistent launch over all pairs, or every
 *   pair's launches (as in fbs_compute_disparity) run in one graph of 1, 2
 *   or 4 concurrent branches.  Scratch: every pair's cost volume at once (sum
 *   of H*W*round_up(D,4)*4 bytes plus statistics).
 *   BF16 / FP16: every pair's tensor-core launches (as in
 *   fbs_compute_disparity) in one graph of 1, 2 or 4 concurrent branches.
 *   Every pair needs D <= 256 and radius <= 24 (FBS_ERR_UNSUPPORTED
 *   otherwise).  Scratch: every pair's 16-bit volume at once (sum of
 *   H*ceil(W/8)*8*Dp*2 bytes, Dp = round_up(D,16) + 16,
 *   plus the packed guide).
 *   A branched graph holds the pairs' addresses: a new set of buffers
 *   captures a new graph (the context keeps up to 32).
 * The first call of a new shape (the list of H, W, C, D, radius, the cost
 * mode and, for the tensor cores, the precision) runs the library's
 * autotuner: it times each schedule plan on the given data and keeps the
 * fastest (recorded in the options' autotune_cache_path file when set, and
 * read back from it by later contexts).  Scratch is owned by ctx.
 * Asynchronous on cuda_stream; the call returns once the work is enqueued.
 */
fbs_status fbs_compute_disparity_batched(fbs_ctx *ctx, int n, const fbs_pair *pairs, void *cuda_stream);

/* The plan the autotuner chose for this batch shape, or -1 if none yet.
 * FP32 (0..6): plans 0..3 persistent, plan = 2 * order + (aggregation CTAs
 * per SM - 1), order 0 = largest pair first, 1 = as given; plans 4..6
 * branched with {1, 2, 4}[plan - 4] branches.  BF16 / FP16 (0..5): plan = 2 * b + s,
 * graph branches {1, 2, 4}[b], window rows per tensor-core pipeline stage
 * s = 0: the kernel's maximum, s = 1: at most 3. */
fbs_status fbs_batch_plan(fbs_ctx *ctx, int n, const fbs_pair *pairs, int *plan);

/* Pin the plan of this batch shape in ctx (numbered as above), skipping the
 * autotuner for it; not written to the autotune cache file.
 * FBS_ERR_INVALID_ARG for a plan outside the context's precision's range. */
fbs_status fbs_batch_set_plan(fbs_ctx *ctx, int n, const fbs_pair *pairs, int plan);

/*
 * fbs_compute_disparity_noalloc -- the whole path without allocating device
 * memory.  The paper has no counterpart: this is an interface variant for
 * callers that cannot call cudaMalloc once they run, such as a plugin inside
 * a host application that owns all device memory through its own allocator,
 * or a real-time loop whose memory budget is fixed at start-up and which may
 * not take an allocation (or the synchronisation cudaMalloc/cudaFree can
 * imply) in the middle of processing.
 *
 * Arguments and results are those of fbs_compute_disparity (FP32 precision
 * only; the context supplies the cost mode, the default stream and the error
 * message).  The context's scratch is not used: the per-pixel block
 * statistics and the cost volume are kept in one file-scope device array of
 * FBS_NOALLOC_MAX_COST_BYTES bytes that is part of the library's device code,
 * so every GPU that loads it holds the array until the process exits (with
 * CUDA's default lazy module loading, from the first call of this entry point
 * on that GPU).
 *   - Limit: H * W * (4 * round_up(D, 4) + 20) bytes (block statistics
 *     20 bytes a pixel, cost volume 4 * round_up(D, 4) bytes a pixel, the
 *     four parts each rounded up to 256 bytes) must fit in
 *     FBS_NOALLOC_MAX_COST_BYTES, e.g. 640x480 with D <= 20 or 320x240 with
 *     D <= 104.  Larger requests return FBS_ERR_INVALID_ARG with the sizes in
 *     fbs_last_error() and launch nothing.
 *   - CUDA context: the context's device is made current (as every entry
 *     point does) and the call then works in the CUDA context current on the
 *     calling thread -- the device's primary context, or a driver-API context
 *     of that device the caller has pushed.  Each call looks up the array's
 *     address in that CUDA context (cudaGetSymbolAddress, a host-side lookup
 *     that allocates nothing; with lazy module loading the first lookup in a
 *     CUDA context also loads the library's device code there, so make one
 *     call before any stream capture) and launches there.
 *   - Sharing: all calls in one CUDA context use the same array, which keeps
 *     the last call's contents.  Nothing in it has to start at zero: each
 *     call writes every element it later reads.  Calls whose kernels overlap
 *     on the GPU (different streams or host threads) race on the array; issue
 *     them on one stream.
 *   - Errors and accounting are those of fbs_compute_disparity: launch
 *     failures return FBS_ERR_CUDA (FBS_ERR_OOM for an out-of-memory error),
 *     and the kernels count under FBS_KERNEL_COST and FBS_KERNEL_AGG_F32 and
 *     are timed when profiling is on.
 *   - The entry point calls no cudaMalloc, cudaFree or allocating library
 *     routine.
 */
#define FBS_NOALLOC_MAX_COST_BYTES (32u * 1024u * 1024u)

fbs_status fbs_compute_disparity_noalloc(fbs_ctx *ctx, const uint8_t *left, const uint8_t *right,
                                         int H, int W, int C, int D, int radius,
                                         float sigma_s, float sigma_r, float tau,
                                         int32_t *disp_int, float *disp_subpix, void *cuda_stream);

/*
 * Kernel accounting (not a step of the method).  The context counts every
 * kernel it launches, per kind.  With profiling enabled it also brackets each
 * launch with a CUDA event pair recorded on the launch stream, so the device
 * time of each kernel kind can be read back.  fbs_profile(ctx, 1) clears the
 * counters and starts recording; fbs_profile(ctx, 0) stops.  fbs_profile_read
 * synchronises on the recorded events and returns, for one kind, the summed
 * device milliseconds (0 when profiling was off) and the number of kernels of
 * that kind launched since the last fbs_profile(ctx, 1) (every kernel counts,
 * also those a step launches inside one timed scope or a CUDA graph).
 */
typedef enum {
    FBS_KERNEL_COST = 0,        /* cost-volume build, Eq. (1)-(3) / TAD */
    FBS_KERNEL_AGG_F32 = 1,     /* FP32 aggregation + WTA + Eq. (10) */
    FBS_KERNEL_AGG_TC = 2,      /* tensor-core aggregation + WTA + Eq. (10) */
    FBS_KERNEL_OTHER = 3,       /* every other kernel of the library */
    FBS_KERNEL_BATCH = 4,       /* one batch graph (timed as a whole; its kernels count under COST, OTHER, AGG_F32 / AGG_TC) */
    FBS_KERNEL_NET = 5,         /* band form: features, network, loss, optimiser, band planning */
    FBS_KERNEL_KINDS = 6
} fbs_kernel_kind;

fbs_status fbs_profile(fbs_ctx *ctx, int enable);
fbs_status fbs_profile_read(fbs_ctx *ctx, int kind, double *total_ms, long long *launches);

#ifdef __cplusplus
}
#endif

#endif /* FBS_H */
