// BF16 tensor-core kernels of the learned initial guess (a U-Net on the node grid).
//
// Convolutions are implicit GEMMs on NHWC bf16 tensors with FP32 accumulation:
//   forward        Y[m][n]  = sum_k A[m][k] W[k][n],   m = output pixel, k = (kh, kw, c_in), n = c_out
//   data gradient  dX[m][n] = sum_k dY'[m][k] W'[k][n], m = input pixel,  k = (kh, kw, c_out), n = c_in
//   weight grad.   dW[m][n] = sum_k A[k][m] dY[k][n],   m = (kh, kw, c_in), k = output pixel, n = c_out
// The A operand is gathered on the fly (zero padding, stride, and the channel concatenation of
// two tensors); tiles are staged in shared memory and multiplied with mma.sync m16n8k16 bf16.
// Channel counts are multiples of 8 so every 16-byte chunk lies in one (kh, kw) tap and one
// source tensor.
#include <cuda_bf16.h>
#include <cstdint>

#include "unet_impl.cuh"

namespace unk {

namespace {

constexpr int BK = 32;          // GEMM k per shared-memory stage
constexpr int SK = BK + 8;      // padded row (bank-conflict-free 32-bit fragment reads)
constexpr int NTHREADS = 128;   // 4 warps, each a 32 x 32 block of the output tile

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// 8 bf16 values of one source pixel (zero outside the image), channels [c, c + 8) of the
// concatenation [x1 (C1 channels), x2 (C2 channels)].
__device__ __forceinline__ uint4 load8(const ConvArgs &a, int b, int y, int x, int H, int W, int c) {
  if (y < 0 || y >= H || x < 0 || x >= W) return make_uint4(0, 0, 0, 0);
  const size_t pix = ((size_t)b * H + y) * W + x;
  if (c < a.C1) return *reinterpret_cast<const uint4 *>(a.x1 + pix * a.C1 + c);
  return *reinterpret_cast<const uint4 *>(a.x2 + pix * a.C2 + (c - a.C1));
}

// Forward gather: A[m][k0 .. k0+7], m = output pixel, k = (kh * ks + kw) * C + ci.
__device__ __forceinline__ uint4 gather_fwd(const ConvArgs &a, int m, int k0) {
  const int C = a.C1 + a.C2;
  if (m >= a.Pout || k0 >= a.Kf) return make_uint4(0, 0, 0, 0);
  const int tap = k0 / C, ci = k0 - tap * C;
  const int kh = tap / a.ks, kw = tap - kh * a.ks;
  const int xo = m % a.Wout, t = m / a.Wout, yo = t % a.Hout, b = t / a.Hout;
  return load8(a, b, yo * a.stride + kh - a.pad, xo * a.stride + kw - a.pad, a.Hin, a.Win, ci);
}

// Data-gradient gather: A[m][k0 .. k0+7], m = input pixel, k = (kh * ks + kw) * Cout + co:
// dY at the output pixel that tap (kh, kw) of m feeds (zero if none).
__device__ __forceinline__ uint4 gather_dgrad(const ConvArgs &a, int m, int k0) {
  if (m >= a.M || k0 >= a.K) return make_uint4(0, 0, 0, 0);
  const int tap = k0 / a.Cout, co = k0 - tap * a.Cout;
  const int kh = tap / a.ks, kw = tap - kh * a.ks;
  const int xi = m % a.Win, t = m / a.Win, yi = t % a.Hin, b = t / a.Hin;
  const int ys = yi + a.pad - kh, xs = xi + a.pad - kw;
  if (ys < 0 || xs < 0 || ys % a.stride || xs % a.stride) return make_uint4(0, 0, 0, 0);
  const int yo = ys / a.stride, xo = xs / a.stride;
  if (yo >= a.Hout || xo >= a.Wout) return make_uint4(0, 0, 0, 0);
  return *reinterpret_cast<const uint4 *>(a.dy + (((size_t)b * a.Hout + yo) * a.Wout + xo) * a.Cout + co);
}

template <int BM, int BN, int MODE>
__global__ void __launch_bounds__(NTHREADS) k_conv(ConvArgs a) {
  __shared__ __align__(16) __nv_bfloat16 As[BM][SK];
  __shared__ __align__(16) __nv_bfloat16 Bs[BN][SK];
  constexpr int WN = BN / 32;  // warps along n
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp / WN, wn = warp % WN;
  const int g = lane >> 2, tq = lane & 3;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  // k range of this block (split-k over output pixels for the weight gradient)
  int kbeg = 0, kend = a.K;
  if (MODE == MODE_WGRAD) {
    const int per = ((a.K + gridDim.z - 1) / gridDim.z + BK - 1) / BK * BK;
    kbeg = blockIdx.z * per;
    kend = min(a.K, kbeg + per);
  }
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    if (MODE != MODE_WGRAD) {
      // A tile: BM rows x 4 chunks of 8 along k
      for (int c = tid; c < BM * (BK / 8); c += NTHREADS) {
        const int r = c / (BK / 8), kc = (c % (BK / 8)) * 8;
        const uint4 v = MODE == MODE_FWD ? gather_fwd(a, m0 + r, k0 + kc) : gather_dgrad(a, m0 + r, k0 + kc);
        *reinterpret_cast<uint4 *>(&As[r][kc]) = v;
      }
      // B tile from the [N][K] weight copy (k contiguous)
      for (int c = tid; c < BN * (BK / 8); c += NTHREADS) {
        const int r = c / (BK / 8), kc = (c % (BK / 8)) * 8;
        const int n = n0 + r, k = k0 + kc;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (n < a.N && k < a.K) v = *reinterpret_cast<const uint4 *>(a.w + (size_t)n * a.K + k);
        *reinterpret_cast<uint4 *>(&Bs[r][kc]) = v;
      }
    } else {
      // weight gradient: GEMM k = output pixel.  A[m][k] = input gather for pixel k, rows
      // m = (kh, kw, ci) -> 8 consecutive rows per 16-byte chunk, scattered into column k.
      for (int c = tid; c < (BM / 8) * BK; c += NTHREADS) {
        const int kk = c % BK, rc = (c / BK) * 8;
        const int p = k0 + kk, row = m0 + rc;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (p < kend) v = gather_fwd(a, p, row);  // forward A element (pixel p, k = row)
        const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
        for (int j = 0; j < 8; ++j) As[rc + j][kk] = e[j];
      }
      for (int c = tid; c < (BN / 8) * BK; c += NTHREADS) {
        const int kk = c % BK, nc = (c / BK) * 8;
        const int p = k0 + kk, n = n0 + nc;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (p < kend && n < a.N) v = *reinterpret_cast<const uint4 *>(a.dy + (size_t)p * a.Cout + n);
        const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
        for (int j = 0; j < 8; ++j) Bs[nc + j][kk] = e[j];
      }
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < BK; ks += 16) {
      uint32_t af[2][4], bfr[4][2];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int r = wm * 32 + mt * 16 + g;
        af[mt][0] = *reinterpret_cast<const uint32_t *>(&As[r][ks + tq * 2]);
        af[mt][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][ks + tq * 2]);
        af[mt][2] = *reinterpret_cast<const uint32_t *>(&As[r][ks + tq * 2 + 8]);
        af[mt][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][ks + tq * 2 + 8]);
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int n = wn * 32 + nt * 8 + g;
        bfr[nt][0] = *reinterpret_cast<const uint32_t *>(&Bs[n][ks + tq * 2]);
        bfr[nt][1] = *reinterpret_cast<const uint32_t *>(&Bs[n][ks + tq * 2 + 8]);
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
          mma_bf16(acc[mt][nt], af[mt][0], af[mt][1], af[mt][2], af[mt][3], bfr[nt][0], bfr[nt][1]);
    }
    __syncthreads();
  }
  // epilogue
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = m0 + wm * 32 + mt * 16 + g + h * 8;
        const int n = n0 + wn * 32 + nt * 8 + tq * 2;
        if (m >= a.M) continue;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int nn = n + e;
          if (nn >= a.N) continue;
          float v = acc[mt][nt][2 * h + e];
          if (MODE == MODE_FWD) {
            if (nn < a.Nreal) v += a.bias[nn];
            if (a.relu) v = fmaxf(v, 0.f);
            if (a.y32) a.y32[(size_t)m * a.N + nn] = v;
            else a.y[(size_t)m * a.N + nn] = __float2bfloat16(v);
          } else if (MODE == MODE_DGRAD) {
            // accumulate into the FP32 gradient of the concatenated input's two parts
            float *d = nn < a.C1 ? &a.dx1[(size_t)m * a.C1 + nn] : &a.dx2[(size_t)m * a.C2 + (nn - a.C1)];
            *d = a.dacc ? *d + v : v;
          } else {
            atomicAdd(&a.dw[(size_t)m * a.N + nn], v);
          }
        }
      }
}

template <int BM, int BN, int MODE>
cudaError_t launch_conv_t(const ConvArgs &a, int splits, cudaStream_t st) {
  dim3 g((a.M + BM - 1) / BM, (a.N + BN - 1) / BN, MODE == MODE_WGRAD ? splits : 1);
  k_conv<BM, BN, MODE><<<g, NTHREADS, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_conv(const ConvArgs &a, int mode, int splits, cudaStream_t st) {
  const bool narrow = a.N <= 32;
  if (mode == MODE_FWD) return narrow ? launch_conv_t<128, 32, MODE_FWD>(a, 1, st) : launch_conv_t<64, 64, MODE_FWD>(a, 1, st);
  if (mode == MODE_DGRAD) return narrow ? launch_conv_t<128, 32, MODE_DGRAD>(a, 1, st) : launch_conv_t<64, 64, MODE_DGRAD>(a, 1, st);
  return narrow ? launch_conv_t<128, 32, MODE_WGRAD>(a, splits, st) : launch_conv_t<64, 64, MODE_WGRAD>(a, splits, st);
}

// ------------------------------------------------------------------------------------------
// elementwise and reduction kernels

// dPre = dOut * (out > 0) for ReLU layers (relu = 0: plain copy), converted to bf16; eight
// consecutive elements per thread (n8 = n / 8, n a multiple of 8: whole 8-channel groups).
// Backward of a layer's output stage: dpre = dout (FP32) masked by out > 0 for ReLU layers,
// rounded to bf16 (the operand of the weight and data gradients), and db[c] += sum over pixels
// of dpre[p][c] for c < Creal (C = channel stride, a multiple of 8, at most 256), in one pass.
// A thread takes one 16-byte group of 8 channels of a pixel-strided set of rows (a warp reads
// whole rows: contiguous bytes); the block adds its rows up in shared memory and makes one
// atomic add per channel.
__global__ void __launch_bounds__(256) k_relu_bias_bwd(const float *dout, const __nv_bfloat16 *out,
                                                       __nv_bfloat16 *dpre, float *db, int P, int C, int Creal,
                                                       int relu) {
  const int G = C / 8, rows = 256 / G;
  const int g = threadIdx.x % G, r = threadIdx.x / G;
  float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (r < rows)
    for (int p = blockIdx.x * rows + r; p < P; p += gridDim.x * rows) {
      const size_t i = (size_t)p * G + g;
      const float4 d0 = reinterpret_cast<const float4 *>(dout)[2 * i], d1 = reinterpret_cast<const float4 *>(dout)[2 * i + 1];
      float v[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
      if (relu) {
        const uint4 o = reinterpret_cast<const uint4 *>(out)[i];
        const __nv_bfloat16 *ob = reinterpret_cast<const __nv_bfloat16 *>(&o);
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (!(__bfloat162float(ob[e]) > 0.f)) v[e] = 0.f;
      }
      uint32_t pk[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
        pk[e] = *reinterpret_cast<const uint32_t *>(&h);
        s[2 * e] += __low2float(h);
        s[2 * e + 1] += __high2float(h);
      }
      reinterpret_cast<uint4 *>(dpre)[i] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
  __shared__ float sh[256][9];
#pragma unroll
  for (int e = 0; e < 8; ++e) sh[threadIdx.x][e] = s[e];
  __syncthreads();
  if ((int)threadIdx.x < Creal) {
    const int c = threadIdx.x, gg = c / 8, e = c % 8;
    float t = 0.f;
    for (int rr = 0; rr < rows; ++rr) t += sh[rr * G + gg][e];
    atomicAdd(&db[c], t);
  }
}

cudaError_t launch_relu_bias_bwd(const float *dout, const __nv_bfloat16 *out, __nv_bfloat16 *dpre, float *db, int P,
                                 int C, int Creal, int relu, cudaStream_t st) {
  if (C % 8 || C > 256 || Creal > C || (relu && !out)) return cudaErrorInvalidValue;
  const int rows = 256 / (C / 8);
  k_relu_bias_bwd<<<std::max(1, std::min(152 * 4, (P + rows - 1) / rows)), 256, 0, st>>>(dout, out, dpre, db, P, C,
                                                                                         Creal, relu);
  return cudaGetLastError();
}

// The output stage of the layer feeding the 1x1 head (d0), fed straight by the head's output
// gradient: g[p][c] = sum_o dyh[p][o] wd[c][o] (the head's data gradient, 8 outputs, never
// stored), then the ReLU mask by the layer's output, bf16 rounding into dpre and the bias
// gradient, in one pass.  Mapping and reduction as k_relu_bias_bwd; the head's 8 x C weights
// in shared memory as FP32 (padded rows), the sum over o in order in FP32.
__global__ void __launch_bounds__(256) k_head_relu_bias_bwd(const __nv_bfloat16 *dyh, const __nv_bfloat16 *wd,
                                                               const __nv_bfloat16 *out, __nv_bfloat16 *dpre,
                                                               float *db, int P, int C, int Creal) {
  // rows of 9 floats: the four channel groups a warp's threads read at once fall in distinct banks
  __shared__ float ws[64 * 9];
  for (int i = threadIdx.x; i < 8 * C; i += blockDim.x) ws[(i / 8) * 9 + i % 8] = __bfloat162float(wd[i]);
  __syncthreads();
  const int G = C / 8, rows = 256 / G;
  const int g = threadIdx.x % G, r = threadIdx.x / G;
  float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (r < rows)
    for (int p = blockIdx.x * rows + r; p < P; p += gridDim.x * rows) {
      const size_t i = (size_t)p * G + g;
      const uint4 q = reinterpret_cast<const uint4 *>(dyh)[p];
      const __nv_bfloat16 *qh = reinterpret_cast<const __nv_bfloat16 *>(&q);
      float d[8];
#pragma unroll
      for (int o = 0; o < 8; ++o) d[o] = __bfloat162float(qh[o]);
      const uint4 ov = reinterpret_cast<const uint4 *>(out)[i];
      const __nv_bfloat16 *ob = reinterpret_cast<const __nv_bfloat16 *>(&ov);
      float v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        // volatile: read in the loop (conflict-free), not hoisted into 64 registers, which would
        // halve the blocks an SM holds and the loads in flight
        const volatile float *w = ws + (8 * g + e) * 9;
        float t = 0.f;
#pragma unroll
        for (int o = 0; o < 8; ++o) t = fmaf(d[o], w[o], t);
        v[e] = __bfloat162float(ob[e]) > 0.f ? t : 0.f;
      }
      uint32_t pk[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
        pk[e] = *reinterpret_cast<const uint32_t *>(&h);
        s[2 * e] += __low2float(h);
        s[2 * e + 1] += __high2float(h);
      }
      reinterpret_cast<uint4 *>(dpre)[i] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
  __shared__ float sh[256][9];
#pragma unroll
  for (int e = 0; e < 8; ++e) sh[threadIdx.x][e] = s[e];
  __syncthreads();
  if ((int)threadIdx.x < Creal) {
    const int c = threadIdx.x, gg = c / 8, e = c % 8;
    float t = 0.f;
    for (int rr = 0; rr < rows; ++rr) t += sh[rr * G + gg][e];
    atomicAdd(&db[c], t);
  }
}

cudaError_t launch_head_relu_bias_bwd(const __nv_bfloat16 *dyh, const __nv_bfloat16 *wd, const __nv_bfloat16 *out,
                                      __nv_bfloat16 *dpre, float *db, int P, int C, int Creal, cudaStream_t st) {
  if (C % 8 || C > 64 || Creal > C) return cudaErrorInvalidValue;
  const int rows = 256 / (C / 8);
  k_head_relu_bias_bwd<<<std::max(1, std::min(152 * 4, (P + rows - 1) / rows)), 256, 0, st>>>(dyh, wd, out, dpre, db,
                                                                                              P, C, Creal);
  return cudaGetLastError();
}

// Node-aligned bilinear upsampling of NHWC bf16: (h, w) -> (2h - 1, 2w - 1); one 16-byte group
// of 8 channels per thread (C a multiple of 8), 32-bit indices (host-checked).
__global__ void k_upsample(const __nv_bfloat16 *in, __nv_bfloat16 *out, int B, int h, int w, int C) {
  const unsigned H = 2 * h - 1, W = 2 * w - 1, G = C / 8;
  const unsigned n = (unsigned)B * H * W * G;
  const uint4 *src = reinterpret_cast<const uint4 *>(in);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned g = i % G, t = i / G, x = t % W, t2 = t / W, y = t2 % H, b = t2 / H;
    const unsigned y0 = y >> 1, y1 = (y + 1) >> 1, x0 = x >> 1, x1 = (x + 1) >> 1;
    const uint4 q[4] = {src[((b * h + y0) * w + x0) * G + g], src[((b * h + y0) * w + x1) * G + g],
                        src[((b * h + y1) * w + x0) * G + g], src[((b * h + y1) * w + x1) * G + g]};
    const __nv_bfloat16 *hq = reinterpret_cast<const __nv_bfloat16 *>(q);
    uint32_t pk[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float v[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int c = 2 * e + k;
        v[k] = 0.25f * (__bfloat162float(hq[c]) + __bfloat162float(hq[8 + c]) + __bfloat162float(hq[16 + c]) +
                        __bfloat162float(hq[24 + c]));
      }
      const __nv_bfloat162 hv = __floats2bfloat162_rn(v[0], v[1]);
      pk[e] = *reinterpret_cast<const uint32_t *>(&hv);
    }
    reinterpret_cast<uint4 *>(out)[i] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
  }
}

cudaError_t launch_upsample(const __nv_bfloat16 *in, __nv_bfloat16 *out, int B, int h, int w, int C, cudaStream_t st) {
  const size_t n = (size_t)B * (2 * h - 1) * (2 * w - 1) * (C / 8);
  if (C % 8 || n >= (1u << 31)) return cudaErrorInvalidValue;
  k_upsample<<<(unsigned)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 152 * 16)), 256, 0, st>>>(in, out, B, h,
                                                                                                      w, C);
  return cudaGetLastError();
}

// Transpose of the upsampling on FP32 gradients: dc[Y][X] = sum of fine gradients weighted by
// the interpolation weights of node (Y, X) (the coarse tensor's only consumer is the upsampling,
// so this is its whole gradient); four channels (one float4) per thread.
__global__ void k_upsample_bwd(const float *dfine, float *dcoarse, int B, int h, int w, int C) {
  const int H = 2 * h - 1, W = 2 * w - 1, G = C / 4;
  const unsigned n = (unsigned)B * h * w * G;
  const float4 *src = reinterpret_cast<const float4 *>(dfine);
  float4 *dst = reinterpret_cast<float4 *>(dcoarse);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned g = i % G, t = i / G, X = t % w, t2 = t / w, Y = t2 % h, b = t2 / h;
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int dy = -1; dy <= 1; ++dy) {
      const int y = 2 * (int)Y + dy;
      if (y < 0 || y >= H) continue;
      const float wy = dy == 0 ? 1.f : 0.5f;
      for (int dx = -1; dx <= 1; ++dx) {
        const int x = 2 * (int)X + dx;
        if (x < 0 || x >= W) continue;
        const float wt = wy * (dx == 0 ? 1.f : 0.5f);
        const float4 f = src[(((unsigned)b * H + y) * W + x) * G + g];
        s.x += wt * f.x; s.y += wt * f.y; s.z += wt * f.z; s.w += wt * f.w;
      }
    }
    dst[i] = s;
  }
}

cudaError_t launch_upsample_bwd(const float *dfine, float *dcoarse, int B, int h, int w, int C, cudaStream_t st) {
  const size_t nf = (size_t)B * (2 * h - 1) * (2 * w - 1) * (C / 4), n = (size_t)B * h * w * (C / 4);
  if (C % 4 || nf >= (1u << 31)) return cudaErrorInvalidValue;
  k_upsample_bwd<<<(unsigned)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 152 * 16)), 256, 0, st>>>(
      dfine, dcoarse, B, h, w, C);
  return cudaGetLastError();
}

// Mean-squared-error loss on the first `nc` of `ld` output channels; writes dL/dy and
// accumulates the loss sum (double) into loss[0].
__global__ void k_mse(const float *y, const float *t, float *dy, size_t P, int ld, int nc, double scale, double *loss) {
  double s = 0.0;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
    for (int c = 0; c < ld; ++c) {
      float g = 0.f;
      if (c < nc) {
        const float d = y[p * ld + c] - t[p * nc + c];
        s += (double)d * d;
        g = (float)(2.0 * scale) * d;
      }
      dy[p * ld + c] = g;
    }
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s * scale);
}

cudaError_t launch_mse(const float *y, const float *t, float *dy, size_t P, int ld, int nc, double *loss,
                       cudaStream_t st) {
  const double scale = 1.0 / ((double)P * nc);
  k_mse<<<(unsigned)std::min<size_t>((P + 255) / 256, 2048), 256, 0, st>>>(y, t, dy, P, ld, nc, scale, loss);
  return cudaGetLastError();
}

// Adam (Kingma & Ba) on FP32 master parameters.
__global__ void k_adam(float *p, const float *g, float *m, float *v, size_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

cudaError_t launch_adam(float *p, const float *g, float *m, float *v, size_t n, float lr, int step, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, 1e-8f, c1, c2);
  return cudaGetLastError();
}

// bf16 operand copies of the layers' FP32 master weights w[kh][kw][ci][co], every layer in one
// launch (a grid-stride loop over the concatenated copies; the layer of an index found by a
// scan of the 12 starts):
//   wf[co][(kh, kw, ci)]  (forward B operand, k contiguous)
//   wd[ci][(kh, kw, co)]  (data-gradient B operand)
//   wdf[ci][(2 - kh, 2 - kw, co)]  (the same with the taps reversed: the weights of the data
//                         gradient written as a forward convolution of dY, stride 1)
// co is padded to cop (zero rows) so that every operand dimension is a multiple of 8.
__global__ void k_weight_copies(WeightCopies c) {
  const size_t total = c.start[c.n];
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    int l = 0;
    while (g >= c.start[l + 1]) ++l;
    const WeightCopy &L = c.l[l];
    const size_t i = g - c.start[l];
    const int taps = L.ks * L.ks;
    const int o = i % L.cop;
    size_t t = i / L.cop;
    const int ch = t % L.ci;
    const int tap = t / L.ci;
    const float v = o < L.co ? L.w[((size_t)tap * L.ci + ch) * L.co + o] : 0.f;
    const __nv_bfloat16 bv = __float2bfloat16(v);
    L.wf[(size_t)o * taps * L.ci + (size_t)tap * L.ci + ch] = bv;
    L.wd[(size_t)ch * taps * L.cop + (size_t)tap * L.cop + o] = bv;
    L.wdf[(size_t)ch * taps * L.cop + (size_t)(taps - 1 - tap) * L.cop + o] = bv;
  }
}

cudaError_t launch_weight_copies(WeightCopies c, cudaStream_t st) {
  if (c.n <= 0 || c.n > kMaxWeightCopies) return cudaErrorInvalidValue;
  c.start[0] = 0;
  for (int l = 0; l < c.n; ++l)
    c.start[l + 1] = c.start[l] + (size_t)c.l[l].ks * c.l[l].ks * c.l[l].ci * c.l[l].cop;
  const size_t n = c.start[c.n];
  k_weight_copies<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, st>>>(c);
  return cudaGetLastError();
}

// Weight gradient in the padded [(kh, kw, ci)][cop] layout -> master layout [(kh, kw, ci)][co].
__global__ void k_unpad_grad(const float *gp, float *g, size_t rows, int co, int cop) {
  const size_t n = rows * co;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    g[i] = gp[(i / co) * cop + i % co];
}

cudaError_t launch_unpad_grad(const float *gp, float *g, size_t rows, int co, int cop, cudaStream_t st) {
  const size_t n = rows * co;
  k_unpad_grad<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, st>>>(gp, g, rows, co, cop);
  return cudaGetLastError();
}

// 1x1 convolution to 8 FP32 output channels (the network head; memory-bound: C bf16 in and
// 8 floats out per pixel): one pixel per thread, its C input channels (C % 8 == 0, C <= 64)
// read as 16-byte groups, the 8 x C bf16 weights ([N][K] rows, the padded rows zero) and the
// bias held in shared memory as FP32, FP32 accumulation in channel order, then the bias.
__global__ void __launch_bounds__(256) k_conv1x1_f32(const __nv_bfloat16 *x, const __nv_bfloat16 *w,
                                                     const float *bias, int Nreal, int C, int P, float *y) {
  __shared__ float ws[8 * 64];
  __shared__ float bs[8];
  for (int i = threadIdx.x; i < 8 * C; i += blockDim.x) ws[i] = __bfloat162float(w[i]);
  if (threadIdx.x < 8) bs[threadIdx.x] = (int)threadIdx.x < Nreal ? bias[threadIdx.x] : 0.f;
  __syncthreads();
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const uint4 *src = reinterpret_cast<const uint4 *>(x + (size_t)p * C);
    for (int g = 0; g < C / 8; ++g) {
      const uint4 q = src[g];
      const __nv_bfloat16 *hq = reinterpret_cast<const __nv_bfloat16 *>(&q);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float v = __bfloat162float(hq[e]);
        const int c = 8 * g + e;
#pragma unroll
        for (int o = 0; o < 8; ++o) acc[o] = fmaf(v, ws[o * C + c], acc[o]);
      }
    }
    float4 *dst = reinterpret_cast<float4 *>(y + (size_t)p * 8);
    dst[0] = make_float4(acc[0] + bs[0], acc[1] + bs[1], acc[2] + bs[2], acc[3] + bs[3]);
    dst[1] = make_float4(acc[4] + bs[4], acc[5] + bs[5], acc[6] + bs[6], acc[7] + bs[7]);
  }
}

bool conv1x1_f32_supported(const ConvArgs &a) {
  return a.ks == 1 && a.stride == 1 && a.pad == 0 && a.y32 && a.N == 8 && a.C2 == 0 && a.C1 % 8 == 0 &&
         a.C1 > 0 && a.C1 <= 64 && a.Nreal <= 8;
}

cudaError_t launch_conv1x1_f32(const ConvArgs &a, cudaStream_t st) {
  if (!conv1x1_f32_supported(a)) return cudaErrorInvalidValue;
  const int blocks = std::max(1, std::min((a.Pout + 255) / 256, 152 * 8));
  k_conv1x1_f32<<<blocks, 256, 0, st>>>(a.x1, a.w, a.bias, a.Nreal, a.C1, a.Pout, a.y32);
  return cudaGetLastError();
}

// Backward of the 1x1 head (C <= 64 input channels, 8 output channels): memory-bound, on the
// CUDA cores.  Weight gradient dw[c][o] += sum over pixels of x[p][c] dy[p][o]: a block stages
// 128 pixels of x and dy in shared memory as FP32 (every thread loading several 16-byte groups
// at once) and thread (o, c) accumulates its entry over the block's pixels (a warp reads 32
// consecutive channels of one pixel and one broadcast dy value), then one atomic add per entry.
constexpr int K1_TP = 128;

__global__ void __launch_bounds__(512) k_conv1x1_wgrad(const __nv_bfloat16 *x, int C, const __nv_bfloat16 *dy, int P,
                                                       float *dw) {
  __shared__ float xs[K1_TP][65];
  __shared__ float ds[K1_TP][8];
  const int tid = threadIdx.x, c = tid % C, o = tid / C, G = C / 8;
  float acc = 0.f;
  for (int p0 = blockIdx.x * K1_TP; p0 < P; p0 += gridDim.x * K1_TP) {
    // K1_TP * G groups over blockDim = 8 C = 64 G threads: K1_TP / 64 per thread, issued before
    // any is used
    constexpr int per = K1_TP / 64;
    uint4 q[per];
#pragma unroll
    for (int k = 0; k < per; ++k) {
      q[k] = make_uint4(0u, 0u, 0u, 0u);
      const int i = tid + k * blockDim.x, pp = i / G, g = i - pp * G;
      if (p0 + pp < P) q[k] = *reinterpret_cast<const uint4 *>(x + (size_t)(p0 + pp) * C + 8 * g);
    }
#pragma unroll
    for (int k = 0; k < per; ++k) {
      const int i = tid + k * blockDim.x, pp = i / G, g = i - pp * G;
      const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&q[k]);
#pragma unroll
      for (int e = 0; e < 8; ++e) xs[pp][8 * g + e] = __bfloat162float(h[e]);
    }
    for (int i = tid; i < K1_TP; i += blockDim.x) {
      uint4 q = make_uint4(0u, 0u, 0u, 0u);
      if (p0 + i < P) q = *reinterpret_cast<const uint4 *>(dy + (size_t)(p0 + i) * 8);
      const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&q);
#pragma unroll
      for (int e = 0; e < 8; ++e) ds[i][e] = __bfloat162float(h[e]);
    }
    __syncthreads();
#pragma unroll 8
    for (int pp = 0; pp < K1_TP; ++pp) acc = fmaf(xs[pp][c], ds[pp][o], acc);
    __syncthreads();
  }
  atomicAdd(&dw[c * 8 + o], acc);
}

bool conv1x1_bwd_supported(const ConvArgs &a) {
  return a.ks == 1 && a.stride == 1 && a.pad == 0 && a.Cout == 8 && a.C2 == 0 && a.C1 % 8 == 0 && a.C1 >= 8 &&
         a.C1 <= 64;
}

cudaError_t launch_conv1x1_wgrad(const ConvArgs &a, const __nv_bfloat16 *dy, float *dw, cudaStream_t st) {
  if (!conv1x1_bwd_supported(a)) return cudaErrorInvalidValue;
  const int blocks = std::max(1, std::min((a.Pout + K1_TP - 1) / K1_TP, 152 * 4));
  k_conv1x1_wgrad<<<blocks, 8 * a.C1, 0, st>>>(a.x1, a.C1, dy, a.Pout, dw);
  return cudaGetLastError();
}

__global__ void k_f32_to_bf16(const float *a, __nv_bfloat16 *b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16(a[i]);
}

cudaError_t launch_f32_to_bf16(const float *a, __nv_bfloat16 *b, size_t n, cudaStream_t st) {
  k_f32_to_bf16<<<(unsigned)std::min<size_t>((n + 255) / 256, 8192), 256, 0, st>>>(a, b, n);
  return cudaGetLastError();
}

}  // namespace unk
