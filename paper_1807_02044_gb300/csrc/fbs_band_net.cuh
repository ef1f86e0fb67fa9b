// Internal declarations of the band-proposal network (the learned band form):
// its geometry, parameter layout and the launchers of its kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fbs {
namespace bnet {

constexpr int kLayers = 6;
constexpr int kFeat = 6;        // features per quarter pixel
constexpr int kFeatPad = 8;     // channels of the first layer's input in memory
constexpr int kWidth = 32;      // hidden channels
constexpr int kOut = 2;         // o0, z
constexpr int kOutPad = 8;      // channels of the output gradient in memory
constexpr int kHeadN = 16;      // MMA N of the last layer (smallest legal N for M = 128)

// Per layer: true channel counts, padded counts in memory, MMA shapes.
__host__ __device__ constexpr int cin(int l) { return l == 0 ? kFeat : kWidth; }
__host__ __device__ constexpr int cout(int l) { return l == kLayers - 1 ? kOut : kWidth; }
__host__ __device__ constexpr int cin_pad(int l) { return l == 0 ? kFeatPad : kWidth; }
__host__ __device__ constexpr int cout_pad(int l) { return l == kLayers - 1 ? kOutPad : kWidth; }
__host__ __device__ constexpr int fwd_n(int l) { return l == kLayers - 1 ? kHeadN : kWidth; }
// K of a 3x3 implicit GEMM over `ch` input channels, in core matrices of 8
// (an even count: one MMA consumes K = 16 = two core matrices).
__host__ __device__ constexpr int k_cores(int ch) { return ((9 * ch / 8) + 1) & ~1; }
// Offset of layer l's weights [3][3][cin][cout] (then its bias) in the flat vector.
__host__ __device__ constexpr int param_offset(int l)
{
    int o = 0;
    for (int j = 0; j < l; ++j) o += 9 * cin(j) * cout(j) + cout(j);
    return o;
}
constexpr int kParams = param_offset(kLayers);

// Packed BF16 weight images, the shared-memory B operand of each MMA
// ([K/8][N][8] elements): forward image of layer l (K over (tap, input
// channel), N = output channels) and data-gradient image of layer l >= 1
// (K over (tap, output channel), N = input channels).
__host__ __device__ constexpr int fwd_image_elems(int l) { return k_cores(cin_pad(l)) * fwd_n(l) * 8; }
__host__ __device__ constexpr int dgrad_image_elems(int l) { return l == 0 ? 0 : k_cores(cout_pad(l)) * cin(l) * 8; }
__host__ __device__ constexpr int fwd_image_offset(int l)
{
    int o = 0;
    for (int j = 0; j < l; ++j) o += fwd_image_elems(j) + dgrad_image_elems(j);
    return o;
}
__host__ __device__ constexpr int dgrad_image_offset(int l) { return fwd_image_offset(l) + fwd_image_elems(l); }
constexpr int kImageElems = fwd_image_offset(kLayers);

// Epilogue of a convolution launch.
enum ConvMode {
    kConvReluBf16 = 0,   // out = relu(acc + bias), BF16 [P][N]
    kConvLinearF32 = 1,  // out = acc + bias, FP32 [P][nout]
    kConvMaskBf16 = 2,   // out = acc * (mask > 0), BF16 [P][N]  (data gradient through a ReLU)
};

// 3x3 convolution, zero padding, of in [P][cin_ch] (P = Hq*Wq quarter pixels,
// row-major) with a packed image of N output channels.  flip: gather the
// neighbour at -offset (data gradient).  err: device word set on a timeout.
cudaError_t launch_conv3x3(int cin_ch, int n, const __nv_bfloat16* in, const __nv_bfloat16* image,
                           const float* bias, const __nv_bfloat16* mask, void* out, int nout, int Hq, int Wq,
                           int flip, int mode, int* err, int num_sms, cudaStream_t stream);
// Weight and bias gradient of layer l: sum over pixels of X[p + offset] G[p],
// X [P][cin_pad(l)], G [P][cout_pad(l)]; written into grad (flat vector).
// On the tensor cores; err: device word set on a timeout.
size_t wgrad_partial_floats(int Hq, int Wq);
cudaError_t launch_wgrad(int l, const __nv_bfloat16* X, const __nv_bfloat16* G, int Hq, int Wq, float* partial,
                         float* grad, int* err, int num_sms, cudaStream_t stream);
// Loss of readings B6 and its gradient G6 [P][kOutPad] (BF16); per-block loss
// sums in loss_partial (loss_blocks(P) floats), reduced into *loss (sum / P).
int loss_blocks(int P);
cudaError_t launch_loss(const float* out, const int32_t* estar, const int32_t* label_int, const float* label_sub,
                        int H, int W, int D, int half_band, __nv_bfloat16* G6, float* loss_partial, float* loss,
                        cudaStream_t stream);
cudaError_t launch_adam(float* theta, float* m, float* v, const float* grad, int n, float lr, float c1, float c2,
                        cudaStream_t stream);
cudaError_t launch_pack_images(const float* theta, __nv_bfloat16* images, cudaStream_t stream);

}  // namespace bnet
}  // namespace fbs
