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
          float4 t = *dst;
          t.x += v[4 * g]; t.y += v[4 * g + 1]; t.z += v[4 * g + 2]; t.w += v[4 * g + 3];
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

int tmem_cols_for(int n) {
  int c = 32;
  while (c < n) c <<= 1;
  return c;
}

}  // namespace

size_t conv_tc_smem(int BN) { return 1024 + (size_t)TC_STAGES * (TC_BM * 128 + (size_t)BN * 128); }

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
