// Internal declarations of the learned-initial-guess network kernels (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>

namespace unk {

enum { MODE_FWD = 0, MODE_DGRAD = 1, MODE_WGRAD = 2 };

// One implicit-GEMM convolution launch (see unet_kernels.cu for the three GEMM shapes).
struct ConvArgs {
  int M, N, K;                    // GEMM sizes of this launch
  int Pout, Kf;                   // output pixels B*Hout*Wout; forward reduction ks*ks*(C1+C2)
  int Bn, Hin, Win, Hout, Wout, ks, stride, pad;
  int C1, C2, Cout;               // input channels (two concatenated tensors), padded output channels
  const __nv_bfloat16 *x1, *x2;   // NHWC inputs
  const __nv_bfloat16 *w;         // [N][K] bf16 operand (forward: wf, data gradient: wd)
  const __nv_bfloat16 *dy;        // NHWC output gradient (bf16), channel stride Cout
  const float *bias;               // Nreal entries (the padded output channels get no bias)
  int Nreal, relu;
  __nv_bfloat16 *y;               // forward output, bf16, channel stride N
  float *y32;                     // or FP32 (network head)
  float *dx1, *dx2;               // data gradient of the two input parts (FP32, accumulated)
  float *dw;                      // weight gradient [M][N] (FP32, atomically accumulated)
  int dsplit;                     // data gradient as a forward convolution of dY (halo / tile kernel): output
                                  // channels [0, dsplit) go to dx1, the rest to dx2
  int dacc;                       // data gradient: 1 = add into dx1 / dx2, 0 = overwrite them (the
                                  // first contribution of the backward pass)
};

cudaError_t launch_conv(const ConvArgs &a, int mode, int splits, cudaStream_t st);
// tcgen05 / TMEM path (forward and data gradient with 16 <= N <= 256, N % 16 == 0)
bool conv_tc_supported(const ConvArgs &a, int mode);
cudaError_t launch_conv_tc(const ConvArgs &a, int mode, int *err, cudaStream_t st);
// tcgen05 weight gradient (MN-major operands from NHWC; 32 <= N <= 128, N % 32 == 0): adds into a.dw
bool wgrad_tc_supported(const ConvArgs &a);
cudaError_t launch_wgrad_tc(const ConvArgs &a, int *err, cudaStream_t st);
// TMA-fed tcgen05 path (forward 3x3 stride-1 convolutions whose input parts have a multiple
// of 32 channels): tensor maps of the two input parts and of the weight matrix
struct ConvMaps {
  CUtensorMap x1, x2, w;
};
bool conv_tma_supported(const ConvArgs &a, int mode);
int make_conv_maps(const ConvArgs &a, int Bmax, ConvMaps *m);
cudaError_t launch_conv_tma(const ConvArgs &a, const ConvMaps &m, int *err, cudaStream_t st);
// the same kernel as the data gradient of a stride-2 layer, split by output parity (a describes a
// stride-1 convolution of dY on its own grid with the data-gradient weights; output on Hf x Wf)
cudaError_t launch_conv_tma_parity(const ConvArgs &a, const ConvMaps &m, int Hf, int Wf, int *err, cudaStream_t st);
// TMA-fed tcgen05 weight gradient (3x3, stride 1 or 2, input parts of a multiple of 32 channels,
// 32 <= N <= 128, N % 32 == 0): tensor maps of the two input parts and of dY (in ConvMaps::w);
// adds into a.dw
bool wgrad_tma_supported(const ConvArgs &a);
int make_wgrad_maps(const ConvArgs &a, int Bmax, ConvMaps *m);
cudaError_t launch_wgrad_tma(const ConvArgs &a, const ConvMaps &m, int *err, cudaStream_t st);
// halo variant (3x3 stride 1, the weight matrix resident in shared memory, <= 72 KB)
bool conv_halo_supported(const ConvArgs &a, int mode);
int make_halo_maps(const ConvArgs &a, int Bmax, ConvMaps *m);
cudaError_t launch_conv_halo(const ConvArgs &a, const ConvMaps &m, int *err, cudaStream_t st);
// FP32-output 1x1 convolution to 8 channels (the head) on the CUDA cores
bool conv1x1_f32_supported(const ConvArgs &a);
cudaError_t launch_conv1x1_f32(const ConvArgs &a, cudaStream_t st);
// ReLU mask, bf16 rounding of the output gradient and the bias gradient in one pass
cudaError_t launch_relu_bias_bwd(const float *dout, const __nv_bfloat16 *out, __nv_bfloat16 *dpre, float *db, int P,
                                 int C, int Creal, int relu, cudaStream_t st);
// the output stage of the layer feeding the head, fed by the head's output gradient dyh (8
// channels): the head's data gradient, ReLU mask, bf16 rounding and bias gradient in one pass
cudaError_t launch_head_relu_bias_bwd(const __nv_bfloat16 *dyh, const __nv_bfloat16 *wd, const __nv_bfloat16 *out,
                                      __nv_bfloat16 *dpre, float *db, int P, int C, int Creal, cudaStream_t st);
// weight gradient of the 1x1 head (C1 <= 64 input channels, 8 padded output channels) on the CUDA
// cores (its data gradient: launch_head_relu_bias_bwd)
bool conv1x1_bwd_supported(const ConvArgs &a);
cudaError_t launch_conv1x1_wgrad(const ConvArgs &a, const __nv_bfloat16 *dy, float *dw, cudaStream_t st);
cudaError_t launch_upsample(const __nv_bfloat16 *in, __nv_bfloat16 *out, int B, int h, int w, int C, cudaStream_t st);
cudaError_t launch_upsample_bwd(const float *dfine, float *dcoarse, int B, int h, int w, int C, cudaStream_t st);
cudaError_t launch_mse(const float *y, const float *t, float *dy, size_t P, int ld, int nc, double *loss,
                       cudaStream_t st);
cudaError_t launch_adam(float *p, const float *g, float *m, float *v, size_t n, float lr, int step, cudaStream_t st);
// the bf16 operand copies (wf, wd, wdf) of every layer's FP32 weights, in one launch
constexpr int kMaxWeightCopies = 12;
struct WeightCopy {
  const float *w;
  __nv_bfloat16 *wf, *wd, *wdf;
  int ks, ci, co, cop;
};
struct WeightCopies {
  WeightCopy l[kMaxWeightCopies];
  size_t start[kMaxWeightCopies + 1];  // filled by launch_weight_copies
  int n;
};
cudaError_t launch_weight_copies(WeightCopies c, cudaStream_t st);
cudaError_t launch_unpad_grad(const float *gp, float *g, size_t rows, int co, int cop, cudaStream_t st);
cudaError_t launch_f32_to_bf16(const float *a, __nv_bfloat16 *b, size_t n, cudaStream_t st);

}  // namespace unk
