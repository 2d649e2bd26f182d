// tcgen05 (5th-generation tensor core) path of the learned-guess convolutions on sm_103a.
//
// Implicit-GEMM convolution, one CTA per 128-row output tile:
//   * four warps gather the A tile (128 rows x 64 k of bf16, im2col on the fly, zero padding)
//     and the B tile (N rows x 64 k of the [N][K] weight copy) into shared memory with
//     cp.async, in the 128-byte-swizzled K-major layout the tensor core reads; two k blocks
//     are in flight while the tensor core works on a third;
//   * one thread issues tcgen05.mma (kind::f16, bf16 x bf16 -> fp32, M = 128, N = tile width,
//     K = 16 per instruction) with the accumulator in tensor memory (TMEM), and tcgen05.commit
//     arrives on an mbarrier per shared-memory stage, which releases that stage for refilling;
//   * the epilogue reads the accumulator back with tcgen05.ld (each warp its 32 TMEM lanes)
//     and applies bias + ReLU (forward) or accumulates the data gradient (FP32).
// Every mbarrier wait is bounded; on a timeout the kernel records an error flag, frees its
// TMEM and returns.
#include <cuda_bf16.h>
#include <cstdint>

#include "unet_impl.cuh"

namespace unk {

namespace {

constexpr int TC_BM = 128;        // tile rows = TMEM lanes
constexpr int TC_BK = 64;         // bf16 per 128-byte row
constexpr int TC_STAGES = 3;
constexpr int TC_THREADS = 128;
constexpr long kWaitLimit = 1L << 22;  // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  for (long it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of 128 bytes,
// 8-row groups 1024 bytes apart (stride-dimension offset); the leading-dimension offset is
// unused for this layout.  Bits: [0,14) address >> 4, [16,30) LBO >> 4, [32,46) SBO >> 4,
// [46,48) descriptor version 1, [61,64) layout 2 = 128-byte swizzle.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)2u << 61;
  return d;
}

// Instruction descriptor of kind::f16: D fp32 (bits 4-5 = 1), A and B bf16 (bits 7-9, 10-12
// = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of 16-byte chunk c (0..7) of row r inside a 1024-byte-aligned swizzled tile
__device__ __forceinline__ uint32_t sw128_off(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

// Per-thread gather plan.  Thread t always fills 16-byte chunk column c = t % 8 of rows
// t / 8 + 16 i (i = 0..7) of the A tile, so the pixel coordinates of those eight rows are
// computed once per CTA; per k block only the tap and channel of column c change.
// Forward: yb, xb = input row and column of tap (0, 0) (in the padding for border pixels;
// rows past the output are marked by a huge negative yb), pb = that tap's input pixel index;
// dgrad: yb, xb, pb = yi + pad, xi + pad, b * Hout.
struct RowPlan {
  int yb[8], xb[8], pb[8];
};

template <int MODE>
__device__ __forceinline__ void plan_rows(const ConvArgs &a, int m0, int tid, RowPlan &P) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + (tid >> 3) + 16 * i;
    if (MODE == MODE_FWD) {
      const int xo = m % a.Wout, t = m / a.Wout, yo = t % a.Hout, b = t / a.Hout;
      const int y0 = yo * a.stride - a.pad, x0 = xo * a.stride - a.pad;
      P.yb[i] = m < a.Pout ? y0 : -(1 << 28);
      P.xb[i] = x0;
      P.pb[i] = (b * a.Hin + y0) * a.Win + x0;
    } else {
      const int xi = m % a.Win, t = m / a.Win, yi = t % a.Hin, b = t / a.Hin;
      P.yb[i] = m < a.M ? yi + a.pad : -(1 << 28);
      P.xb[i] = xi + a.pad;
      P.pb[i] = b * a.Hout;
    }
  }
}

// cp.async the A and B chunks of k block kt into stage tiles sa / sb, then commit one group
template <int MODE>
__device__ __forceinline__ void gather_stage(const ConvArgs &a, const RowPlan &P, int tid, int kt, int BN, uint32_t sa,
                                             uint32_t sb) {
  const int c = tid & 7, r0 = tid >> 3;
  const int k = kt * TC_BK + c * 8;
  if (MODE == MODE_FWD) {
    const int C = a.C1 + a.C2;
    const bool kv = k < a.Kf;
    const int tap = kv ? k / C : 0, ci = k - tap * C;
    const int kh = tap / a.ks, kw = tap - kh * a.ks;
    const int toff = kh * a.Win + kw;
    const __nv_bfloat16 *base = ci < a.C1 ? a.x1 + ci : a.x2 + (ci - a.C1);
    const size_t ch = ci < a.C1 ? a.C1 : a.C2;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const bool v = kv && (unsigned)(P.yb[i] + kh) < (unsigned)a.Hin && (unsigned)(P.xb[i] + kw) < (unsigned)a.Win;
      const __nv_bfloat16 *src = v ? base + (size_t)(P.pb[i] + toff) * ch : a.w;
      cp_async16(sa + sw128_off(r0 + 16 * i, c), src, v);
    }
  } else {
    const bool kv = k < a.K;
    const int tap = kv ? k / a.Cout : 0, co = k - tap * a.Cout;
    const int kh = tap / a.ks, kw = tap - kh * a.ks;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int ys = P.yb[i] - kh, xs = P.xb[i] - kw;
      bool v = kv && ys >= 0 && xs >= 0;
      int yo = ys, xo = xs;
      if (a.stride == 2) {
        v = v && !(ys & 1) && !(xs & 1);
        yo = ys >> 1;
        xo = xs >> 1;
      }
      v = v && yo < a.Hout && xo < a.Wout;
      const __nv_bfloat16 *src = v ? a.dy + ((size_t)(P.pb[i] + yo) * a.Wout + xo) * a.Cout + co : a.w;
      cp_async16(sa + sw128_off(r0 + 16 * i, c), src, v);
    }
  }
  for (int r = r0; r < BN; r += 16) {
    const bool v = r < a.N && k < a.K;
    cp_async16(sb + sw128_off(r, c), v ? (const void *)(a.w + (size_t)r * a.K + k) : (const void *)a.w, v);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int MODE>
__global__ void __launch_bounds__(TC_THREADS) k_conv_tc(ConvArgs a, int BN, int tmem_cols, int *err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned tiles: A stages, then B stages
  const uint32_t base0 = smem_u32(smem_raw);
  const uint32_t base = (base0 + 1023u) & ~1023u;
  const uint32_t a_bytes = TC_BM * 128, b_bytes = (uint32_t)BN * 128;
  __shared__ __align__(8) uint64_t bars[TC_STAGES];
  __shared__ uint32_t tmem_base_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TC_BM;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0)
    for (int s = 0; s < TC_STAGES; ++s) mbar_init(&bars[s], 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  RowPlan P;
  plan_rows<MODE>(a, m0, tid, P);
  const int KT = (a.K + TC_BK - 1) / TC_BK;
  auto stage_a = [&](int kt) { return base + (uint32_t)(kt % TC_STAGES) * a_bytes; };
  auto stage_b = [&](int kt) { return base + TC_STAGES * a_bytes + (uint32_t)(kt % TC_STAGES) * b_bytes; };
  // prologue: k blocks 0 .. STAGES-2 in flight (one cp.async group each, empty past the end)
#pragma unroll
  for (int p = 0; p < TC_STAGES - 1; ++p) {
    if (p < KT) gather_stage<MODE>(a, P, tid, p, BN, stage_a(p), stage_b(p));
    else asm volatile("cp.async.commit_group;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  const uint32_t idesc = idesc_bf16(TC_BM, BN);
  bool ok = true;

  for (int kt = 0; kt < KT; ++kt) {
    // this thread's chunks of block kt have landed; make them visible to the tensor core
    asm volatile("cp.async.wait_group %0;" ::"n"(TC_STAGES - 2) : "memory");
    fence_proxy_async();
    ok = __syncthreads_and(ok);  // every thread's chunks landed, and no wait has timed out
    if (!ok) break;
    if (tid == 0) {
      tc_fence_after();
      const uint32_t sa = stage_a(kt), sb = stage_b(kt);
#pragma unroll
      for (int kk = 0; kk < TC_BK / 16; ++kk) {
        const uint64_t da = sw128_desc(sa + kk * 32), db = sw128_desc(sb + kk * 32);
        const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&bars[kt % TC_STAGES]))
                   : "memory");
    }
    // refill the stage that block kt-1 used, once its MMAs have read it
    const int nk = kt + TC_STAGES - 1;
    if (nk < KT) {
      if (kt >= 1) ok = mbar_wait(&bars[(kt - 1) % TC_STAGES], (uint32_t)(((kt - 1) / TC_STAGES) & 1));
      if (ok) gather_stage<MODE>(a, P, tid, nk, BN, stage_a(nk), stage_b(nk));
      else asm volatile("cp.async.commit_group;" ::: "memory");
    } else {
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  // the last commit covers every MMA issued
  if (ok && KT > 0) {
    const int kl = KT - 1;
    ok = mbar_wait(&bars[kl % TC_STAGES], (uint32_t)((kl / TC_STAGES) & 1));
  }
  ok = __syncthreads_and(ok);
  tc_fence_after();
  if (ok) {
    const int m = m0 + warp * 32 + lane;
    for (int n0 = 0; n0 < BN; n0 += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)n0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m >= a.M) continue;
      float v[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(r[e]);
      if (MODE == MODE_FWD) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          if (n0 + e < a.Nreal) v[e] += a.bias[n0 + e];
          if (a.relu) v[e] = fmaxf(v[e], 0.f);
        }
        if (a.y32) {
          for (int e = 0; e < 16; ++e)
            if (n0 + e < a.N) a.y32[(size_t)m * a.N + n0 + e] = v[e];
        } else {
          // N % 16 == 0: the 16 outputs are one aligned 32-byte run of the row
          uint32_t pk[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
            pk[e] = *reinterpret_cast<const uint32_t *>(&h);
          }
          uint4 *dst = reinterpret_cast<uint4 *>(a.y + (size_t)m * a.N + n0);
          dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
          dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
      } else {
        // channel groups of 4 lie wholly in one input part (C1 % 8 == 0)
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const int n = n0 + 4 * g;
          if (n >= a.N) break;
          float4 *dst = n < a.C1 ? reinterpret_cast<float4 *>(a.dx1 + (size_t)m * a.C1 + n)
                                 : reinterpret_cast<float4 *>(a.dx2 + (size_t)m * a.C2 + (n - a.C1));
          float4 t = make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
          if (a.dacc) {
            const float4 o = *dst;
            t.x += o.x; t.y += o.y; t.z += o.z; t.w += o.w;
          }
          *dst = t;
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

// ------------------------------------------------------------------------------------------
// Weight gradient on tcgen05: dW[m][n] = sum over output pixels k of A[m][k] dY[k][n], with
// m = (kh, kw, c_in) and A[m][k] the input value that tap (kh, kw) of output pixel k reads.
// Both operands are pixel-major in memory (NHWC), so they are staged MN-major: A in 128-byte
// swizzle atoms of 64 m x 8 pixels (one 16-byte chunk = 8 input channels of one source pixel),
// B in 64-byte swizzle atoms of 32 output channels x 8 pixels.  One CTA per 128-row tile of m
// and range of pixels accumulates in TMEM over its whole range (split over the pixels: the K
// dimension), then adds its tile into dW with one FP32 atomic per element.
constexpr int WG_BK = 64;                 // pixels per k block (8 groups of 8)
constexpr int WG_STAGE = 16384;           // bytes of each A and B stage (B sized for N <= 128)
constexpr uint32_t WG_SBO_A = 1024;       // next group of 8 pixels: 8 rows x 128 B
constexpr uint32_t WG_LBO_A = 8 * 1024;   // next 64 m: after the k block's 8 groups
constexpr uint32_t WG_SBO_B = 512;        // next group of 8 pixels: 8 rows x 64 B
constexpr uint32_t WG_LBO_B = 8 * 512;    // next 32 output channels
constexpr int WG_GUARD = 16384;           // beyond the last stage (reads stay inside the CTA's shared memory)

// MN-major shared-memory descriptors: [0,14) address >> 4, [16,30) LBO >> 4 (next atom along
// M / N), [32,46) SBO >> 4 (next group of 8 along K), [46,48) version 1, [61,64) layout
// 2 = 128-byte swizzle / 4 = 64-byte swizzle.
__device__ __forceinline__ uint64_t mn_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)layout << 61;
  return d;
}

// kind::f16, D fp32, A and B bf16, both transposed (MN-major): bits 15 and 16
__host__ __device__ constexpr uint32_t idesc_bf16_mn(int M, int N) { return idesc_bf16(M, N) | (1u << 15) | (1u << 16); }

// cp.async the A and B chunks of pixel block [p0, p0 + 64) into stage tiles sa / sb: thread t
// takes pixel p0 + t / 2 and half of its chunks
__device__ __forceinline__ void gather_wgrad(const ConvArgs &a, int m0, int p0, int tid, uint32_t sa, uint32_t sb) {
  const int r = tid >> 1, half = tid & 1;
  const int p = p0 + r;
  const bool pv = p < a.Pout;
  int yo = 0, xo = 0, b = 0;
  if (pv) {
    xo = p % a.Wout;
    const int t = p / a.Wout;
    yo = t % a.Hout;
    b = t / a.Hout;
  }
  const int C = a.C1 + a.C2;
  const int g = r >> 3, rr = r & 7;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int c = half * 8 + j;  // 16-byte chunk of the 128 m rows
    const int m = m0 + 8 * c;
    const int tap = m / C, ci = m - tap * C;
    const int kh = tap / a.ks, kw = tap - kh * a.ks;
    const int y = yo * a.stride + kh - a.pad, x = xo * a.stride + kw - a.pad;
    const bool v = pv && m < a.M && (unsigned)y < (unsigned)a.Hin && (unsigned)x < (unsigned)a.Win;
    const size_t pix = ((size_t)b * a.Hin + y) * a.Win + x;
    const __nv_bfloat16 *src = !v ? a.x1 : (ci < a.C1 ? a.x1 + pix * a.C1 + ci : a.x2 + pix * a.C2 + (ci - a.C1));
    cp_async16(sa + (uint32_t)(c >> 3) * WG_LBO_A + (uint32_t)g * WG_SBO_A + (uint32_t)rr * 128 +
                   ((uint32_t)((c & 7) ^ rr) << 4),
               src, v);
  }
  const int nb = a.N >> 3, nh = nb >> 1;  // 16-byte chunks of the N output channels
  for (int c = half * nh; c < (half + 1) * nh; ++c) {
    const __nv_bfloat16 *src = pv ? a.dy + (size_t)p * a.Cout + c * 8 : a.dy;
    cp_async16(sb + (uint32_t)(c >> 2) * WG_LBO_B + (uint32_t)g * WG_SBO_B + (uint32_t)rr * 64 +
                   ((uint32_t)((c & 3) ^ ((rr >> 1) & 3)) << 4),
               src, pv);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__global__ void __launch_bounds__(TC_THREADS) k_wgrad_tc(ConvArgs a, int kb_per, int tmem_cols, int *err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t base0 = smem_u32(smem_raw);
  const uint32_t base = (base0 + 1023u) & ~1023u;
  __shared__ __align__(8) uint64_t bars[TC_STAGES];
  __shared__ uint32_t tmem_base_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TC_BM;
  const int KB = (a.Pout + WG_BK - 1) / WG_BK;
  const int kb0 = blockIdx.y * kb_per, kb1 = min(KB, kb0 + kb_per);
  const int KT = max(0, kb1 - kb0);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0)
    for (int s = 0; s < TC_STAGES; ++s) mbar_init(&bars[s], 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  auto stage_a = [&](int kt) { return base + (uint32_t)(kt % TC_STAGES) * (2 * WG_STAGE); };
  auto stage_b = [&](int kt) { return base + (uint32_t)(kt % TC_STAGES) * (2 * WG_STAGE) + WG_STAGE; };
#pragma unroll
  for (int p = 0; p < TC_STAGES - 1; ++p) {
    if (p < KT) gather_wgrad(a, m0, (kb0 + p) * WG_BK, tid, stage_a(p), stage_b(p));
    else asm volatile("cp.async.commit_group;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  const uint32_t idesc = idesc_bf16_mn(TC_BM, a.N);
  bool ok = true;
  for (int kt = 0; kt < KT; ++kt) {
    asm volatile("cp.async.wait_group %0;" ::"n"(TC_STAGES - 2) : "memory");
    fence_proxy_async();
    ok = __syncthreads_and(ok);
    if (!ok) break;
    if (tid == 0) {
      tc_fence_after();
      const uint32_t sa = stage_a(kt), sb = stage_b(kt);
#pragma unroll
      for (int kk = 0; kk < WG_BK / 16; ++kk) {
        const uint64_t da = mn_desc(sa + (uint32_t)(2 * kk) * WG_SBO_A, WG_LBO_A, WG_SBO_A, 2u);
        const uint64_t db = mn_desc(sb + (uint32_t)(2 * kk) * WG_SBO_B, WG_LBO_B, WG_SBO_B, 4u);
        const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&bars[kt % TC_STAGES]))
                   : "memory");
    }
    const int nk = kt + TC_STAGES - 1;
    if (nk < KT) {
      if (kt >= 1) ok = mbar_wait(&bars[(kt - 1) % TC_STAGES], (uint32_t)(((kt - 1) / TC_STAGES) & 1));
      if (ok) gather_wgrad(a, m0, (kb0 + nk) * WG_BK, tid, stage_a(nk), stage_b(nk));
      else asm volatile("cp.async.commit_group;" ::: "memory");
    } else {
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  if (ok && KT > 0) {
    const int kl = KT - 1;
    ok = mbar_wait(&bars[kl % TC_STAGES], (uint32_t)((kl / TC_STAGES) & 1));
  }
  ok = __syncthreads_and(ok);
  tc_fence_after();
  if (ok && KT > 0) {
    const int m = m0 + warp * 32 + lane;
    for (int n0 = 0; n0 < a.N; n0 += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)n0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m < a.M) {
#pragma unroll
        for (int e = 0; e < 16; ++e) atomicAdd(&a.dw[(size_t)m * a.N + n0 + e], __uint_as_float(r[e]));
      }
    }
  } else if (!ok && tid == 0) {
    atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

int tmem_cols_for(int n) {
  int c = 32;
  while (c < n) c <<= 1;
  return c;
}

}  // namespace

size_t conv_tc_smem(int BN) { return 1024 + (size_t)TC_STAGES * (TC_BM * 128 + (size_t)BN * 128); }

size_t wgrad_tc_smem() { return 1024 + (size_t)TC_STAGES * 2 * WG_STAGE + WG_GUARD; }

// weight gradient: input parts of whole 16-byte chunks, output channels in whole 64-byte swizzle
// atoms (32 .. 128, the accumulator's TMEM columns)
bool wgrad_tc_supported(const ConvArgs &a) {
  return a.C1 % 8 == 0 && a.C2 % 8 == 0 && a.N % 32 == 0 && a.N >= 32 && a.N <= 128 && a.Cout == a.N &&
         (a.stride == 1 || a.stride == 2) && a.M > 0 && a.Pout > 0;
}

cudaError_t launch_wgrad_tc(const ConvArgs &a, int *err, cudaStream_t st) {
  const int mt = (a.M + TC_BM - 1) / TC_BM;
  const int KB = (a.Pout + WG_BK - 1) / WG_BK;
  // about two CTAs per SM in all: pixel ranges of whole k blocks
  const int splits = std::max(1, std::min(KB, (2 * 152 + mt - 1) / mt));
  const int kb_per = (KB + splits - 1) / splits;
  const int gy = (KB + kb_per - 1) / kb_per;
  const size_t smem = wgrad_tc_smem();
  cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_wgrad_tc<<<dim3(mt, gy), TC_THREADS, smem, st>>>(a, kb_per, tmem_cols_for(a.N), err);
  return cudaGetLastError();
}

bool conv_tc_supported(const ConvArgs &a, int mode) {
  if (mode == MODE_WGRAD) return false;
  // 16-byte gather chunks must not straddle a tap or the two concatenated inputs
  if (a.C1 % 8 || a.C2 % 8 || a.Cout % 8 || (a.stride != 1 && a.stride != 2)) return false;
  return a.N % 16 == 0 && a.N >= 16 && a.N <= 256;
}

cudaError_t launch_conv_tc(const ConvArgs &a, int mode, int *err, cudaStream_t st) {
  const int BN = a.N;  // whole output width in one tile (multiple of 16, <= 256)
  const size_t smem = conv_tc_smem(BN);
  dim3 g((a.M + TC_BM - 1) / TC_BM);
  if (mode == MODE_FWD) {
    cudaFuncSetAttribute(k_conv_tc<MODE_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_conv_tc<MODE_FWD><<<g, TC_THREADS, smem, st>>>(a, BN, tmem_cols_for(BN), err);
  } else {
    cudaFuncSetAttribute(k_conv_tc<MODE_DGRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_conv_tc<MODE_DGRAD><<<g, TC_THREADS, smem, st>>>(a, BN, tmem_cols_for(BN), err);
  }
  return cudaGetLastError();
}

}  // namespace unk
