/*
 * fbs_band.h -- C ABI of the learned band form of libfbs.
 *
 * The paper closes (Sec. V) with the idea of shrinking the disparity search
 * range of each pixel to cut the cost of filtering the whole cost volume.
 * This form does that with a learned proposal:
 *
 *   1. features:  at quarter resolution (Hq = ceil(H/4), Wq = ceil(W/4),
 *                 Dq = ceil(D/4)) the images are reduced to 4x4 block sums of
 *                 the channel-sum intensity; an unaggregated coarse NCC
 *                 (Eq. (1)-(3) on those planes, cost K = 1 - c) gives per
 *                 quarter pixel the coarse winner e* and six features
 *                 (left intensity, e* / Dq, K(e*), the margin to the best
 *                 non-adjacent e, and the cost steps to e* - 1 and e* + 1);
 *   2. network:   six 3x3 convolutions (6 -> 32 -> 32 -> 32 -> 32 -> 32 -> 2,
 *                 zero padding, ReLU after the first five), BF16 operands on
 *                 the tensor cores with FP32 accumulation, output o0 (the
 *                 correction of e* in quarter disparities) and z (the logit
 *                 of the confidence);
 *   3. band:      full-resolution centre c = 4 (e* + o0) and confidence
 *                 k = 1 / (1 + exp(-z)), taken from the quarter pixel
 *                 (x / 4, y / 4); a pixel with k >= threshold searches only
 *                 [m - h, m + h] clipped to [0, D - 1], m = floor(c + 0.5)
 *                 clamped to [0, D - 1]; every other pixel keeps [0, D - 1];
 *   4. band FBS:  Eq. (6)-(8) for the disparities of each pixel's band only,
 *                 WTA over the band (smallest d on ties) and Eq. (10) when
 *                 both neighbours of the winner lie in the band.
 *
 * The network is trained by the library's own kernels on disparity maps of
 * the plain full-range path: loss per quarter pixel
 *   y huber(c - t) + bce(z, y),
 * t = median subpixel label over the 4x4 block, y = the share of the block's
 * integer labels in [m - h + 1, m + h - 1] for the predicted band centre m
 * (pixels whose band holds the winner and both of its neighbours; y also
 * weights the centre term so that blocks no band can serve are left to the
 * fallback); Adam updates FP32 master weights, which are rounded to BF16 for
 * the MMAs.
 *
 * Conventions are those of fbs.h (status codes, device pointers owned by the
 * caller, asynchronous on the given stream, host-side validation).  The
 * network's weights, optimiser state and activations are owned by the
 * context; a new context starts with fbs_band_net_init(ctx, 0).
 */
#ifndef FBS_BAND_H
#define FBS_BAND_H

#include "fbs.h"

#ifdef __cplusplus
extern "C" {
#endif

#define FBS_BAND_FEATURES 6
#define FBS_BAND_WIDTH 32
#define FBS_BAND_LAYERS 6

/* Number of FP32 parameters: for each layer l = 1..6, W_l as
 * [3][3][Cin_l][Cout_l] (row offset, column offset, input, output channel)
 * followed by b_l [Cout_l]; Cin = (6, 32, 32, 32, 32, 32),
 * Cout = (32, 32, 32, 32, 32, 2). */
size_t fbs_band_net_param_count(void);

/* He-normal weights from a seeded splitmix64 / Box-Muller stream (the last
 * layer scaled by 0.1), zero biases, fresh Adam state. */
fbs_status fbs_band_net_init(fbs_ctx *ctx, uint64_t seed);

/* Copy the FP32 parameters from / to HOST memory (n must equal
 * fbs_band_net_param_count()).  set_params also clears the Adam state. */
fbs_status fbs_band_net_set_params(fbs_ctx *ctx, const float *params, size_t n);
fbs_status fbs_band_net_get_params(fbs_ctx *ctx, float *params, size_t n);

/* Parameters as a little-endian file: 8-byte tag "FBSBAND1", uint32 count,
 * count float32 values. */
fbs_status fbs_band_net_save(fbs_ctx *ctx, const char *path);
fbs_status fbs_band_net_load(fbs_ctx *ctx, const char *path);

/*
 * Step 1 alone: feat (nullable) receives [Hq][Wq][6] float32, estar
 * (nullable) the coarse winner [Hq][Wq] int32.  NCC cost only.
 */
fbs_status fbs_band_features(fbs_ctx *ctx, const uint8_t *left, const uint8_t *right,
                             int H, int W, int C, int D, float *feat, int32_t *estar,
                             void *cuda_stream);

/*
 * Steps 1-3: the network's outputs out_q [Hq][Wq][2] (o0, z; nullable) and
 * the full-resolution centre and confidence [H][W] (each nullable, not all
 * three NULL).
 */
fbs_status fbs_band_net_forward(fbs_ctx *ctx, const uint8_t *left, const uint8_t *right,
                                int H, int W, int C, int D, float *out_q, float *centre,
                                float *conf, void *cuda_stream);

/*
 * One training step on one pair: forward, loss, backward and (when lr > 0)
 * an Adam update (beta1 0.9, beta2 0.999, eps 1e-8) with step size lr.
 * label_int / label_sub: the plain path's disparities of this pair [H][W]
 * (device).  half_band: h of the confidence target.  loss (nullable, HOST)
 * receives the loss and grad (nullable, HOST, param_count floats) the
 * gradient of this step; either makes the call wait for the step to finish.
 */
fbs_status fbs_band_net_train_step(fbs_ctx *ctx, const uint8_t *left, const uint8_t *right,
                                   int H, int W, int C, int D, const int32_t *label_int,
                                   const float *label_sub, int half_band, float lr,
                                   float *loss, float *grad, void *cuda_stream);

/*
 * Parity / debug entry point (not a method step; the paper has no
 * counterpart): the intermediate tensors of the context's last
 * fbs_band_net_forward or fbs_band_net_train_step call, as FP32 copies, so a
 * test can check every layer on its own inputs.  P = ceil(H/4) * ceil(W/4)
 * quarter pixels of that call; both buffers are device memory owned by the
 * caller, channels innermost:
 *   acts (nullable): P * (8 + 5 * 32 + 2) floats -- the network input [P][8]
 *     (the six features rounded to BF16, two zero channels), the hidden
 *     activations Y_1 .. Y_5 [P][32] each (BF16 values), the outputs [P][2];
 *   grads (nullable; only after a training step, else FBS_ERR_INVALID_ARG):
 *     P * (5 * 32 + 8) floats -- for layers 1..5 the BF16 gradient of the loss
 *     with respect to the layer's pre-activation [P][32] each (the gradient
 *     with respect to Y_l masked by its ReLU), then the BF16 gradient with
 *     respect to the outputs [P][8] (two channels used).
 * Returns FBS_ERR_INVALID_ARG (launching nothing) before any such call.
 */
fbs_status fbs_band_net_trace(fbs_ctx *ctx, float *acts, float *grads, void *cuda_stream);

/*
 * The non-learned band source the paper names as future work (Sec. V):
 * reliable feature points suggest the search range of their neighbours.  A
 * quarter pixel is a feature point when its coarse cost margin (feature f3 of
 * step 1) is >= margin_threshold; a pixel whose 5x5 quarter neighbourhood
 * (clipped) holds at least 3 feature points with coarse winners e* spread by
 * at most 2 gets centre 2 (max e* + min e*) (4x the mid-range) and confidence
 * 1, every other pixel confidence 0.  centre, conf: [H][W] float32 (device),
 * to be passed to fbs_compute_disparity_banded with a threshold in (0, 1].
 */
fbs_status fbs_band_feature_points(fbs_ctx *ctx, const uint8_t *left, const uint8_t *right,
                                   int H, int W, int C, int D, float margin_threshold,
                                   float *centre, float *conf, void *cuda_stream);

/*
 * Step 3's band rule on given centre / confidence planes (n elements, device):
 * writes lo[n], hi[n] (device int32).  1 <= half_band <= 512.
 */
fbs_status fbs_band_limits(fbs_ctx *ctx, const float *centre, const float *conf, int n, int D,
                           int half_band, float conf_threshold, int32_t *lo, int32_t *hi,
                           void *cuda_stream);

/*
 * Step 4: band-restricted FBS of one pair (NCC cost, FP32 arithmetic) with
 * the bands given by centre / conf [H][W] (device float32; step 3's rule).
 * Scratch: a full [H][W][round_up(D,4)] float32 cost volume of which only the
 * disparities some aggregation tile needs are computed and read.
 */
fbs_status fbs_compute_disparity_banded(fbs_ctx *ctx, const fbs_pair *pair, const float *centre,
                                        const float *conf, int half_band, float conf_threshold,
                                        void *cuda_stream);

/*
 * Steps 1-4 in one call: the network's proposal followed by the band FBS.
 */
fbs_status fbs_compute_disparity_learned(fbs_ctx *ctx, const fbs_pair *pair, int half_band,
                                         float conf_threshold, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* FBS_BAND_H */
