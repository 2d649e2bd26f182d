// tcgen05 convolutions of the learned-guess network fed by the Tensor Memory Accelerator.
//
// For the 3x3 convolutions of stride 1 or 2 whose input parts have a multiple of 32 channels,
// the GEMM rows are the output pixels in tiles of 16 x 8 pixels of one image (M = 128) and the
// columns all output channels (N <= 128).  The reduction runs over (tap, input part, 32-channel
// chunk) in the order of the weight matrix's K index (tap-major, then the channels of the
// concatenated inputs).  For each chunk one TMA tiled load brings the 16 x 8 input pixels that
// the tap reads (for stride 2 every second pixel, by the load's element strides), 32 channels
// each, into shared memory (64-byte rows, 64-byte swizzle; coordinates outside the image read
// zero, which is the convolution's padding) and one brings the N x 32 weight slice.
//
// The kernel is persistent (a CTA walks tiles blockIdx.x, blockIdx.x + gridDim.x, ...) and warp
// specialised: lane 0 of warp 0 issues the TMA loads into an S-stage ring (mbarriers "full",
// completed by the TMA byte count, and "empty", completed by tcgen05.commit once the MMAs that
// read a stage are done); lane 0 of warp 1 issues tcgen05.mma (kind::f16, K = 16, two per chunk)
// into one of two TMEM accumulators (columns [0, N) and [cols / 2, cols / 2 + N) of a
// power-of-two allocation of at least 2N columns); warps 2-5 drain the other accumulator (tcgen05.ld, bias,
// ReLU, bf16 stores) and hand it back ("acc_empty").  Every wait is bounded and also ends when
// another role has given up; before the CTA leaves, the producer waits for its loads still in
// flight and the MMA thread for its last MMAs, and warp 0 frees the TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstring>

#include "unet_impl.cuh"

namespace unk {

namespace {

constexpr int TM_X = 16, TM_Y = 8;     // output tile (x fastest): 128 GEMM rows
constexpr int TM_CH = 32;              // channels per chunk: 64-byte rows
constexpr int TM_MAXS = 8;             // most pipeline stages
constexpr int TM_THREADS = 192;        // producer warp, MMA warp, 4 epilogue warps
constexpr int TM_NMAX = 128;
constexpr long kTmaWaitLimit = 1L << 22;

__device__ __forceinline__ uint32_t saddr(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ bool try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// wait for the phase of the given parity; false after kTmaWaitLimit polls or once *abort is set
__device__ __forceinline__ bool wait_bounded(uint32_t bar, uint32_t parity, volatile int *abort) {
  for (long it = 0; it < kTmaWaitLimit; ++it) {
    if (try_wait(bar, parity)) return true;
    if (*abort) return false;
  }
  *abort = 1;
  return false;
}

// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle, rows of 64 bytes, 8-row
// groups 512 bytes apart.  Bits: [0,14) address >> 4, [16,30) LBO >> 4 (unused here),
// [32,46) SBO >> 4, [46,48) descriptor version 1, [61,64) layout 4 = 64-byte swizzle.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t a) {
  uint64_t d = 0;
  d |= (uint64_t)((a >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;
  d |= (uint64_t)(512u >> 4) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)4u << 61;
  return d;
}

__host__ __device__ constexpr uint32_t idesc_bf16_tma(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

struct TileGrid {
  int tx, ty, per_img, ntiles;
};

__device__ __forceinline__ void tile_origin(const TileGrid &g, int t, int &x0, int &y0, int &b) {
  b = t / g.per_img;
  const int r = t - b * g.per_img;
  y0 = (r / g.tx) * TM_Y;
  x0 = (r % g.tx) * TM_X;
}

// The tile kernel as the data gradient of a stride-2 3x3 convolution, split by output parity:
// input pixel (2Y + a, 2X + c) receives the taps (kh, kw) with kh = a + 1 and kw = c + 1 (mod 2),
// which read dY at (Y + (a + 1 - kh) / 2, X + (c + 1 - kw) / 2).  So class (a, c) is a stride-1
// convolution of dY on the coarse grid with 1, 2, 2 or 4 taps (each tap's K block of the
// data-gradient weights wd), written at every second input pixel.  The tiles of the four classes
// follow one another in the launch.
struct ParityTaps {
  int on;             // 0: a plain convolution (nine taps, output at the tile's pixels)
  int per_class;      // tiles of one class
  int Hf, Wf;         // the input (fine) grid the gradient is written on
  int n[4];           // taps of class 2 a + c
  int dx[4][4], dy[4][4], tap[4][4];
};

__device__ __forceinline__ void tile_of(const TileGrid &g, const ParityTaps &pt, int t, int &x0, int &y0, int &b,
                                        int &cls) {
  cls = 0;
  if (pt.on) {
    cls = t / pt.per_class;
    t -= cls * pt.per_class;
  }
  tile_origin(g, t, x0, y0, b);
}

__global__ void __launch_bounds__(TM_THREADS) k_conv_tma(const __grid_constant__ CUtensorMap mx1,
                                                         const __grid_constant__ CUtensorMap mx2,
                                                         const __grid_constant__ CUtensorMap mw, ConvArgs a,
                                                         TileGrid tg, ParityTaps pt, int S, int tmem_cols,
                                                         int *err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int BN = a.N;
  const uint32_t base = (saddr(smem_raw) + 1023u) & ~1023u;
  const uint32_t a_bytes = TM_X * TM_Y * 64, st_bytes = a_bytes + (uint32_t)BN * 64;
  __shared__ __align__(8) uint64_t full[TM_MAXS], empty[TM_MAXS], acc_full[2], acc_empty[2], mma_done;
  __shared__ uint32_t tmem_sh;
  __shared__ int abort_sh;
  volatile int *abort = &abort_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_sh)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 32) {
    abort_sh = 0;
    for (int s = 0; s < S; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&empty[s])) : "memory");
    }
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&acc_full[i])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(saddr(&acc_empty[i])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&mma_done)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_sh;

  const int c1 = a.C1 / TM_CH, c2 = a.C2 / TM_CH, per_tap = c1 + c2;
  const int nk = 9 * per_tap;

  if (warp == 0 && lane == 0) {
    // ---- producer: TMA loads of every chunk of every tile of this CTA, in order
    const uint64_t pm1 = reinterpret_cast<uint64_t>(&mx1), pm2 = reinterpret_cast<uint64_t>(&mx2),
                   pmw = reinterpret_cast<uint64_t>(&mw);
    long g = 0;  // chunks issued so far
    for (int t = blockIdx.x; t < tg.ntiles && !*abort; t += gridDim.x) {
      int x0, y0, b, cls;
      tile_of(tg, pt, t, x0, y0, b, cls);
      const int nkt = pt.on ? pt.n[cls] * per_tap : nk;
      for (int k = 0; k < nkt; ++k, ++g) {
        const int s = (int)(g % S);
        const uint32_t use = (uint32_t)(g / S);
        if (use > 0 && !wait_bounded(saddr(&empty[s]), (use - 1) & 1, abort)) break;
        const int i = k / per_tap, q = k - i * per_tap;
        int tap, xs, ys;
        if (pt.on) {
          tap = pt.tap[cls][i];
          xs = x0 + pt.dx[cls][i];
          ys = y0 + pt.dy[cls][i];
        } else {
          tap = i;
          const int kh = tap / 3, kw = tap - kh * 3;
          xs = x0 * a.stride + kw - 1;
          ys = y0 * a.stride + kh - 1;
        }
        const uint64_t mx = q < c1 ? pm1 : pm2;
        const int cc = (q < c1 ? q : q - c1) * TM_CH;
        const uint32_t sa = base + (uint32_t)s * st_bytes, sb = sa + a_bytes, bar = saddr(&full[s]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(st_bytes) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
            ::"r"(sa), "l"(mx), "r"(cc), "r"(xs), "r"(ys), "r"(b), "r"(bar)
            : "memory");
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
            ::"r"(sb), "l"(pmw), "r"(tap * (a.C1 + a.C2) + q * TM_CH), "r"(0), "r"(bar)
            : "memory");
      }
    }
    // loads still in flight: the last min(S, g) issued, one per stage, each the latest on its stage
    volatile int never = 0;
    for (long j = g > S ? g - S : 0; j < g; ++j)
      wait_bounded(saddr(&full[j % S]), (uint32_t)((j / S) & 1), &never);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    const uint32_t idesc = idesc_bf16_tma(TM_X * TM_Y, BN);
    const uint64_t dA0 = sw64_desc(base);
    long g = 0;
    int j = 0;  // tiles of this CTA so far
    bool ok = true;
    for (int t = blockIdx.x; t < tg.ntiles && ok; t += gridDim.x, ++j) {
      const int ab = j & 1;
      if (j >= 2 && !(ok = wait_bounded(saddr(&acc_empty[ab]), (uint32_t)(((j >> 1) - 1) & 1), abort))) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t acc_t = tmem + (uint32_t)(ab * (tmem_cols >> 1));
      const int nkt = pt.on ? pt.n[t / pt.per_class] * per_tap : nk;
      for (int k = 0; k < nkt; ++k, ++g) {
        const int s = (int)(g % S);
        if (!(ok = wait_bounded(saddr(&full[s]), (uint32_t)((g / S) & 1), abort))) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // stage s: A at dA0 + s * st_bytes, B a_bytes after it; the second K = 16 step 32 bytes on
        const uint64_t da = dA0 + (uint64_t)((uint32_t)s * (st_bytes >> 4));
        asm volatile(
            "{\n .reg .pred p, q;\n .reg .b64 a1, b1, b0;\n"
            " setp.ne.b32 p, %3, 0;\n setp.eq.b32 q, %3, %3;\n"
            " add.s64 b0, %1, %4;\n add.s64 a1, %1, 2;\n add.s64 b1, b0, 2;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, b0, %2, p;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], a1, b1, %2, q;\n}\n" ::"r"(acc_t),
            "l"(da), "r"(idesc), "r"(k > 0 ? 1u : 0u), "l"((uint64_t)(a_bytes >> 4)));
        commit(saddr(&empty[s]));
      }
      if (ok) commit(saddr(&acc_full[ab]));
    }
    // every MMA issued has finished before the CTA goes on to free the TMEM
    commit(saddr(&mma_done));
    volatile int never = 0;
    wait_bounded(saddr(&mma_done), 0, &never);
  } else if (warp >= 2) {
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 = GEMM rows of the tile
    const int quarter = warp & 3;
    const int m = quarter * 32 + lane;
    int j = 0;
    for (int t = blockIdx.x; t < tg.ntiles; t += gridDim.x, ++j) {
      const int ab = j & 1;
      // every lane waits (acquire); the warp goes on only together, as tcgen05.ld is .aligned
      const bool got = wait_bounded(saddr(&acc_full[ab]), (uint32_t)((j >> 1) & 1), abort);
      if (!__all_sync(0xffffffffu, got)) {
        *abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int x0, y0, b, cls;
      tile_of(tg, pt, t, x0, y0, b, cls);
      int xx = x0 + (m % TM_X), yy = y0 + (m / TM_X), Wo = a.Wout, Ho = a.Hout;
      if (pt.on) {  // class (a, c) of the parity split: every second input pixel
        xx = 2 * xx + (cls & 1);
        yy = 2 * yy + (cls >> 1);
        Wo = pt.Wf;
        Ho = pt.Hf;
      }
      const bool inside = xx < Wo && yy < Ho;
      const size_t pix = ((size_t)b * Ho + yy) * Wo + xx;
      for (int n0 = 0; n0 < BN; n0 += 16) {
        uint32_t r[16];
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ab * (tmem_cols >> 1) + n0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (!inside) continue;
        if (a.dx1) {
          // data gradient (a forward convolution of dY): write (or add) into the FP32 gradient of
          // the input part these 16 channels belong to (dsplit is a multiple of 32)
          const bool p1 = n0 < a.dsplit;
          const int cw = p1 ? a.dsplit : a.N - a.dsplit;
          float4 *dst = reinterpret_cast<float4 *>((p1 ? a.dx1 : a.dx2) + pix * cw + (p1 ? n0 : n0 - a.dsplit));
          float4 o[4];
#pragma unroll
          for (int e = 0; e < 4; ++e)
            o[e] = make_float4(__uint_as_float(r[4 * e]), __uint_as_float(r[4 * e + 1]), __uint_as_float(r[4 * e + 2]),
                               __uint_as_float(r[4 * e + 3]));
          if (a.dacc) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float4 q = dst[e];
              o[e].x += q.x; o[e].y += q.y; o[e].z += q.z; o[e].w += q.w;
            }
          }
#pragma unroll
          for (int e = 0; e < 4; ++e) dst[e] = o[e];
          continue;
        }
        float v[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          v[e] = __uint_as_float(r[e]);
          if (n0 + e < a.Nreal) v[e] += a.bias[n0 + e];
          if (a.relu) v[e] = fmaxf(v[e], 0.f);
        }
        uint32_t pk[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
          pk[e] = *reinterpret_cast<const uint32_t *>(&h);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(a.y + pix * a.N + n0);
        dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      arrive(saddr(&acc_empty[ab]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0 && abort_sh) atomicExch(err, 1);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

// ---- halo variant (tensor path 3): one load per 32-channel chunk serves all nine taps ----------
//
// For 3x3 stride-1 layers whose whole weight matrix fits in shared memory (at most 72 KB), the
// weights are loaded once per CTA and stay resident, and a tile is 8 x 16 output pixels.  Per
// 32-channel chunk four TMA loads (one per 8-channel group, 16-byte rows, no swizzle) bring the
// 10 x 18-pixel halo of the tile; the nine taps are nine windows of it.  In the halo a group
// plane holds pixel (x, y) at (y * 10 + x) * 16 bytes, so the 8 pixels of one output row at one
// tap are a contiguous 128-byte core matrix (8 rows x 16 bytes), the next output row's core
// matrix lies 160 bytes on (SBO) and the next 8 channels one plane slot, 2,944 bytes, on (LBO): an unswizzled
// K-major operand whose start address moves with the tap.  A chunk takes 18 MMAs (9 taps x
// K 32).  The reduction runs chunk by chunk, each chunk tap by tap (the thread-gather and the
// path-2 kernels run tap by tap, each tap over all channels), so the FP32 sums round differently.
constexpr int HX = 8, HY = 16;                   // output tile
constexpr int HW = HX + 2, HH = HY + 2;          // halo
constexpr uint32_t HPLANE = HW * HH * 16;        // one 8-channel group: 2,880 bytes loaded
constexpr uint32_t HPITCH = 2944;                // its slot: rounded up to 128 bytes, as a TMA destination must be
constexpr uint32_t HSTAGE = 4 * HPITCH;          // one 32-channel chunk: 11,776 bytes
constexpr uint32_t HTX = 4 * HPLANE;             // bytes its four loads deliver
constexpr int HSTAGES = 4;
constexpr uint32_t HWMAX = 72 * 1024;            // largest resident weight matrix

// Unswizzled K-major descriptor: core matrices of 8 rows x 16 bytes, LBO between K-adjacent and
// SBO between M/N-adjacent core matrices; layout type 0 (no swizzle), descriptor version 1.
__device__ __forceinline__ uint64_t nosw_desc(uint32_t a, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((a >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1u << 46;
  return d;
}

__device__ __forceinline__ void halo_origin(const TileGrid &g, int t, int &x0, int &y0, int &b) {
  b = t / g.per_img;
  const int r = t - b * g.per_img;
  y0 = (r / g.tx) * HY;
  x0 = (r % g.tx) * HX;
}

__global__ void __launch_bounds__(TM_THREADS) k_conv_halo(const __grid_constant__ CUtensorMap mx1,
                                                          const __grid_constant__ CUtensorMap mx2,
                                                          const __grid_constant__ CUtensorMap mw, ConvArgs a,
                                                          TileGrid tg, int tmem_cols, int *err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int BN = a.N;
  // c8: an 8-channel input (one plane per tile, taps paired into K = 16 MMAs); the weights then
  // as ten unswizzled blocks of 8 K values (the tenth past K = 72: the load's zero fill)
  const bool c8 = a.C1 == 8;
  const int Ctot = a.C1 + a.C2, nkb = c8 ? 10 : 9 * Ctot / TM_CH;  // weight blocks of 32 (8) K values
  const uint32_t wblk = (uint32_t)BN * (c8 ? 16 : 64), wbytes = (uint32_t)nkb * wblk;
  const uint32_t wbase = (saddr(smem_raw) + 1023u) & ~1023u, hbase = wbase + wbytes;
  __shared__ __align__(8) uint64_t wfull, full[HSTAGES], empty[HSTAGES], acc_full[2], acc_empty[2], mma_done;
  __shared__ uint32_t tmem_sh;
  __shared__ int abort_sh;
  volatile int *abort = &abort_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_sh)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 32) {
    abort_sh = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&wfull)) : "memory");
    for (int s = 0; s < HSTAGES; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&empty[s])) : "memory");
    }
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&acc_full[i])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(saddr(&acc_empty[i])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&mma_done)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_sh;
  const int c1 = a.C1 / TM_CH, nch = c8 ? 1 : Ctot / TM_CH;

  if (warp == 0) {
    // ---- producer warp: the weight matrix once, then the halo of every chunk of every tile;
    // lane 0 waits for a free stage and posts its byte count, lanes 0-3 load one 8-channel
    // group each
    const uint64_t pm1 = reinterpret_cast<uint64_t>(&mx1), pm2 = reinterpret_cast<uint64_t>(&mx2),
                   pmw = reinterpret_cast<uint64_t>(&mw);
    const uint32_t wb = saddr(&wfull);
    if (lane == 0) {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(wb), "r"(wbytes) : "memory");
      for (int i = 0; i < nkb; ++i)
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
            ::"r"(wbase + (uint32_t)i * wblk), "l"(pmw), "r"(i * (c8 ? 8 : TM_CH)), "r"(0), "r"(wb)
            : "memory");
    }
    long g = 0;
    bool go = true;
    for (int t = blockIdx.x; t < tg.ntiles && go; t += gridDim.x) {
      int x0, y0, b;
      halo_origin(tg, t, x0, y0, b);
      for (int c = 0; c < nch; ++c, ++g) {
        const int s = (int)(g % HSTAGES);
        const uint32_t use = (uint32_t)(g / HSTAGES), bar = saddr(&full[s]);
        int ok = 1;
        if (lane == 0) {
          ok = !*abort && (use == 0 || wait_bounded(saddr(&empty[s]), (use - 1) & 1, abort));
          if (ok)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(c8 ? HPLANE : HTX)
                         : "memory");
        }
        if (!__shfl_sync(0xffffffffu, ok, 0)) {
          go = false;
          break;
        }
        if (lane < (c8 ? 1 : 4))
          asm volatile(
              "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
              ::"r"(hbase + (uint32_t)s * HSTAGE + (uint32_t)lane * HPITCH), "l"(c < c1 ? pm1 : pm2),
                "r"((c < c1 ? c : c - c1) * TM_CH + 8 * lane), "r"(x0 - 1), "r"(y0 - 1), "r"(b), "r"(bar)
              : "memory");
      }
    }
    if (lane == 0) {
      volatile int never = 0;
      wait_bounded(wb, 0, &never);
      for (long j = g > HSTAGES ? g - HSTAGES : 0; j < g; ++j)
        wait_bounded(saddr(&full[j % HSTAGES]), (uint32_t)((j / HSTAGES) & 1), &never);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    const uint32_t idesc = idesc_bf16_tma(HX * HY, BN);
    const uint64_t dH0 = nosw_desc(hbase, HPITCH, HW * 16), dW0 = sw64_desc(wbase);
    const uint64_t w_tap = (uint64_t)(((uint32_t)nch * wblk) >> 4);
    bool ok = wait_bounded(saddr(&wfull), 0, abort);
    long g = 0;
    int j = 0;
    for (int t = blockIdx.x; t < tg.ntiles && ok; t += gridDim.x, ++j) {
      const int ab = j & 1;
      if (j >= 2 && !(ok = wait_bounded(saddr(&acc_empty[ab]), (uint32_t)(((j >> 1) - 1) & 1), abort))) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t acc_t = tmem + (uint32_t)(ab * (tmem_cols >> 1));
      for (int c = 0; c < nch; ++c, ++g) {
        const int s = (int)(g % HSTAGES);
        if (!(ok = wait_bounded(saddr(&full[s]), (uint32_t)((g / HSTAGES) & 1), abort))) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (c8) {
          // taps (2q, 2q + 1) form one K = 16 step: the second core matrix along K is the window
          // of tap 2q + 1, (its offset - tap 2q's) bytes on (the LBO of that MMA; the windows
          // overlap in memory, which the reads allow); the weights' K blocks 512 B apart
          const uint32_t sa = hbase + (uint32_t)s * HSTAGE;
#pragma unroll
          for (int q = 0; q < 5; ++q) {
            const int t0 = 2 * q, t1 = 2 * q + 1;
            const uint32_t o0 = (uint32_t)((t0 / 3) * HW + t0 % 3) * 16;
            // the padding tap (K 72..79, zero weights) reads tap 8's window again: loaded,
            // finite data (stale shared memory could hold NaN, and NaN x 0 is NaN)
            const uint32_t o1 = t1 < 9 ? (uint32_t)((t1 / 3) * HW + t1 % 3) * 16 : o0;
            const uint64_t da = nosw_desc(sa + o0, o1 - o0, HW * 16);
            const uint64_t db = nosw_desc(wbase + (uint32_t)t0 * wblk, wblk, 128);
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc_t),
                "l"(da), "l"(db), "r"(idesc), "r"(q > 0 ? 1u : 0u));
          }
          commit(saddr(&empty[s]));
          continue;
        }
        // descriptors advance by constants: tap (kh, kw) = window (kh * 10 + kw) * 16 bytes on, its
        // weight block nch * wblk bytes on; the second K = 16 step two planes / 32 bytes on
        const uint64_t da0 = dH0 + (uint64_t)((uint32_t)s * (HSTAGE >> 4));
        const uint64_t db0 = dW0 + (uint64_t)((uint32_t)c * (wblk >> 4));
        const uint32_t first = c > 0 ? 1u : 0u;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap)
          asm volatile(
              "{\n .reg .pred p, q;\n .reg .b64 a1, b1;\n"
              " setp.ne.b32 p, %4, 0;\n setp.eq.b32 q, %4, %4;\n"
              " add.s64 a1, %1, %5;\n add.s64 b1, %2, 2;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], a1, b1, %3, q;\n}\n" ::"r"(acc_t),
              "l"(da0 + (uint64_t)((tap / 3) * HW + tap % 3)), "l"(db0 + (uint64_t)tap * w_tap), "r"(idesc),
              "r"(tap > 0 ? 1u : first), "n"((2 * HPITCH) >> 4));
        commit(saddr(&empty[s]));
      }
      if (ok) commit(saddr(&acc_full[ab]));
    }
    commit(saddr(&mma_done));
    volatile int never = 0;
    wait_bounded(saddr(&mma_done), 0, &never);
  } else if (warp >= 2) {
    // ---- epilogue: TMEM lane m = GEMM row = output pixel (x0 + m % 8, y0 + m / 8)
    const int quarter = warp & 3;
    const int m = quarter * 32 + lane;
    int j = 0;
    for (int t = blockIdx.x; t < tg.ntiles; t += gridDim.x, ++j) {
      const int ab = j & 1;
      const bool got = wait_bounded(saddr(&acc_full[ab]), (uint32_t)((j >> 1) & 1), abort);
      if (!__all_sync(0xffffffffu, got)) {
        *abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int x0, y0, b;
      halo_origin(tg, t, x0, y0, b);
      const int xx = x0 + (m % HX), yy = y0 + (m / HX);
      const bool inside = xx < a.Wout && yy < a.Hout;
      const size_t pix = ((size_t)b * a.Hout + yy) * a.Wout + xx;
      for (int n0 = 0; n0 < BN; n0 += 16) {
        uint32_t r[16];
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ab * (tmem_cols >> 1) + n0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (!inside) continue;
        if (a.dx1) {
          // data gradient: write (or add) into the FP32 gradient of the input part these 16
          // channels belong to (dsplit is a multiple of 32: a group of 16 never straddles the parts)
          const bool p1 = n0 < a.dsplit;
          const int cw = p1 ? a.dsplit : a.N - a.dsplit;
          float4 *dst = reinterpret_cast<float4 *>((p1 ? a.dx1 : a.dx2) + pix * cw + (p1 ? n0 : n0 - a.dsplit));
          float4 o[4];
#pragma unroll
          for (int e = 0; e < 4; ++e)
            o[e] = make_float4(__uint_as_float(r[4 * e]), __uint_as_float(r[4 * e + 1]), __uint_as_float(r[4 * e + 2]),
                               __uint_as_float(r[4 * e + 3]));
          if (a.dacc) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float4 q = dst[e];
              o[e].x += q.x; o[e].y += q.y; o[e].z += q.z; o[e].w += q.w;
            }
          }
#pragma unroll
          for (int e = 0; e < 4; ++e) dst[e] = o[e];
          continue;
        }
        float v[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          v[e] = __uint_as_float(r[e]);
          if (n0 + e < a.Nreal) v[e] += a.bias[n0 + e];
          if (a.relu) v[e] = fmaxf(v[e], 0.f);
        }
        uint32_t pk[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
          pk[e] = *reinterpret_cast<const uint32_t *>(&h);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(a.y + pix * a.N + n0);
        dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      arrive(saddr(&acc_empty[ab]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0 && abort_sh) atomicExch(err, 1);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

// ---- weight gradient fed by TMA (tensor path 3) ------------------------------------------------
//
// dW[m][n] = sum over output pixels k of A[m][k] dY[k][n], m = (tap, input channel) in the order of
// the weight matrix, n = output channel.  Both operands are pixel-major in memory (NHWC), so they
// enter the tensor core MN-major: a TMA box of 32 channels x a segment of 64 or 128 output pixels
// (P columns x R rows of one image; for stride 2 the box spans 2P x 2R input pixels traversed
// with element strides 2) lands as a stack of 64-byte-swizzle atoms (32 channels x 8 pixels, 512
// bytes each), a "slice".  A CTA owns a group of Cg 32-channel input slices for all nine taps and
// a range of pixel segments; per segment it loads 9 Cg input slices (one per tap and slice: the
// window the tap reads) and N / 32 slices of dY.  The input slices are stored in the order of m,
// so any four consecutive ones form the A operand of one M = 128 MMA (atoms one slice apart: the
// descriptor's leading offset); the accumulators of all ceil(9 Cg / 4) such tiles stay in TMEM
// over the CTA's whole pixel range and are added into dW once at the end (FP32 atomics).  A last
// tile that runs past the 9 Cg slices reads the slices after them (or the guard after the ring):
// those TMEM rows are discarded.  Warp roles: warp 0 loads (each lane its boxes), lane 0 of warp 1
// issues the MMAs, all four warps drain TMEM; every wait is bounded.
constexpr int WT_THREADS = 128;
constexpr int WT_MAXS = 6;

struct WgPlan {
  int sc;              // channels per input slice: 32 (64-byte swizzle) or 8 (no swizzle)
  int pix;             // output pixels per segment: 64 or 128 (four or eight K = 16 steps)
  uint32_t slice;      // bytes of one input slice: sc channels x pix pixels of bf16
  uint32_t bslice;     // bytes of one dY slice: 32 channels x pix pixels
  int a_slots;         // input slots of a stage before the dY slices (9 Cg, or whole tiles for sc 8)
  int P, R;            // segment: P output columns x R output rows (P * R = pix)
  int tx, per_img;     // segments per output row band, per image
  int units;           // segments of the batch
  int c1;              // input slices of part 1 (part 2 follows)
  int Cg;              // input slices per channel group (gridDim.y groups)
  int tiles;           // M = 128 tiles: ceil(9 Cg sc / 128)
  int nb;              // dY slices: N / 32
  int S;               // pipeline stages
  int per_cta;         // segments per CTA
};

// MN-major shared-memory descriptor: [0,14) address >> 4, [16,30) LBO >> 4, [32,46) SBO >> 4,
// version 1, layout 4 (64-byte swizzle: atoms of 32 channels x 8 pixels, 512 bytes) or 0 (no
// swizzle: core matrices of 8 channels x 8 pixels, 128 bytes); which offset steps along M and
// which along K depends on the layout (see the MMA issuer)
__device__ __forceinline__ uint64_t mn_desc(uint32_t a, uint32_t lbo, uint32_t sbo, uint32_t layout) {
  uint64_t d = 0;
  d |= (uint64_t)((a >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)layout << 61;
  return d;
}

template <int SC>
__global__ void __launch_bounds__(WT_THREADS) k_wgrad_tma(const __grid_constant__ CUtensorMap mx1,
                                                          const __grid_constant__ CUtensorMap mx2,
                                                          const __grid_constant__ CUtensorMap mdy, ConvArgs a,
                                                          WgPlan p, int tmem_cols, int *err) {
  // K = 16 pixels: two 8-pixel groups of the input operand (512-byte atoms for SC = 32, 128-byte
  // core matrices for SC = 8) and of dY (512-byte atoms); in descriptor address units (16 bytes)
  constexpr uint32_t KA = SC == 32 ? 64 : 16, KB = 64;
  constexpr int SPT = 128 / SC;  // input slices per M = 128 tile
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t base = (saddr(smem_raw) + 1023u) & ~1023u;
  const int na = 9 * p.Cg;
  const uint32_t boff0 = (uint32_t)p.a_slots * p.slice;
  const uint32_t st_bytes = boff0 + (uint32_t)p.nb * p.bslice;
  const uint32_t tx_bytes = (uint32_t)na * p.slice + (uint32_t)p.nb * p.bslice;
  __shared__ __align__(8) uint64_t full[WT_MAXS], empty[WT_MAXS], mma_done;
  __shared__ uint32_t tmem_sh;
  __shared__ int abort_sh;
  volatile int *abort = &abort_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int grp = blockIdx.y;
  const int u0 = blockIdx.x * p.per_cta, u1 = min(p.units, u0 + p.per_cta);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_sh)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 32) {
    abort_sh = 0;
    for (int s = 0; s < p.S; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&empty[s])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&mma_done)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_sh;
  bool mma_ok = false;

  if (warp == 0) {
    // ---- producer warp: lane 0 waits for a free stage and posts its byte count, then each lane
    // issues its boxes of the segment (box j: input slice (tap, cg) for j < 9 Cg, else dY slice
    // j - 9 Cg); per lane at most two boxes, whose map, channel, tap offset and destination
    // offset do not change from segment to segment
    const uint64_t pm1 = reinterpret_cast<uint64_t>(&mx1), pm2 = reinterpret_cast<uint64_t>(&mx2),
                   pmd = reinterpret_cast<uint64_t>(&mdy);
    const int nbox = na + p.nb;
    uint64_t bmap[2] = {pmd, pmd};
    int bc[2] = {0, 0}, bdx[2] = {0, 0}, bdy[2] = {0, 0}, bs[2] = {1, 1};
    uint32_t boff[2] = {0, 0};
    int mine = 0;
    for (int j = lane; j < nbox && mine < 2; j += 32, ++mine) {
      if (j < na) {
        const int tap = j / p.Cg, cg = j - tap * p.Cg, kh = tap / 3, kw = tap - kh * 3;
        const int sl = grp * p.Cg + cg;
        boff[mine] = (uint32_t)j * p.slice;
        bmap[mine] = sl < p.c1 ? pm1 : pm2;
        bc[mine] = (sl < p.c1 ? sl : sl - p.c1) * SC;
        bdx[mine] = kw - 1;
        bdy[mine] = kh - 1;
        bs[mine] = a.stride;
      } else {
        boff[mine] = boff0 + (uint32_t)(j - na) * p.bslice;
        bc[mine] = 32 * (j - na);
      }
    }
    long g = 0;
    for (int u = u0; u < u1; ++u, ++g) {
      const int s = (int)(g % p.S);
      const uint32_t use = (uint32_t)(g / p.S), bar = saddr(&full[s]);
      int ok = 1;
      if (lane == 0) {
        if (use > 0) ok = wait_bounded(saddr(&empty[s]), (use - 1) & 1, abort);
        if (ok)
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tx_bytes) : "memory");
      }
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      const int b = u / p.per_img, r = u - b * p.per_img;
      const int y0 = (r / p.tx) * p.R, x0 = (r % p.tx) * p.P;
      const uint32_t sa = base + (uint32_t)s * st_bytes;
      for (int i = 0; i < mine; ++i)
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
            ::"r"(sa + boff[i]), "l"(bmap[i]), "r"(bc[i]), "r"(x0 * bs[i] + bdx[i]), "r"(y0 * bs[i] + bdy[i]), "r"(b),
              "r"(bar)
            : "memory");
    }
    // loads still in flight: the last min(S, g) stages posted, each the latest on its stage
    if (lane == 0) {
      volatile int never = 0;
      for (long j = g > p.S ? g - p.S : 0; j < g; ++j)
        wait_bounded(saddr(&full[j % p.S]), (uint32_t)((j / p.S) & 1), &never);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: every tile accumulates over every segment of the CTA.  The descriptors of
    // stage 0 are built once; a stage, a tile (SPT slices) and a K step of 16 pixels only add to
    // the address field (bytes >> 4; addresses stay below 2^18).
    const uint32_t idesc = idesc_bf16_tma(128, a.N) | (1u << 15) | (1u << 16);  // A and B MN-major
    // 64-byte swizzle: LBO = next slice along M, SBO = next 8 pixels along K; no swizzle (the
    // canonical layout of 8 x 16-byte core matrices): LBO = next 8 pixels along K, SBO = next
    // slice along M
    const uint64_t dA0 = SC == 32 ? mn_desc(base, p.slice, 512u, 4u) : mn_desc(base, 128u, p.slice, 0u);
    const uint64_t dB0 = mn_desc(base + boff0, p.bslice, 512u, 4u);
    const uint64_t d_stage = st_bytes >> 4, d_tile = ((uint32_t)SPT * p.slice) >> 4;
    long g = 0;
    bool ok = true;
    for (int u = u0; u < u1; ++u, ++g) {
      const int s = (int)(g % p.S);
      if (!(ok = wait_bounded(saddr(&full[s]), (uint32_t)((g / p.S) & 1), abort))) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t db = dB0 + (uint64_t)s * d_stage;
      uint64_t da = dA0 + (uint64_t)s * d_stage;
      uint32_t dt = tmem;
      const uint32_t first = g > 0 ? 1u : 0u;
      // four K = 16 steps per block; a 128-pixel segment takes two blocks
      const int blocks = p.pix / 64;
      for (int t = 0; t < p.tiles; ++t, da += d_tile, dt += (uint32_t)a.N)
        for (int h = 0; h < blocks; ++h)
          asm volatile(
              "{\n .reg .pred p, q;\n .reg .b64 a1, a2, a3, b1, b2, b3;\n"
              " setp.ne.b32 p, %4, 0;\n setp.eq.b32 q, %4, %4;\n"
              " add.s64 a1, %1, %5;\n add.s64 a2, %1, %6;\n add.s64 a3, %1, %7;\n"
              " add.s64 b1, %2, %8;\n add.s64 b2, %2, %9;\n add.s64 b3, %2, %10;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], a1, b1, %3, q;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], a2, b2, %3, q;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], a3, b3, %3, q;\n}\n" ::"r"(dt),
              "l"(da + (uint64_t)(h * 4 * KA)), "l"(db + (uint64_t)(h * 4 * KB)), "r"(idesc), "r"(h > 0 ? 1u : first),
              "n"(KA), "n"(2 * KA), "n"(3 * KA), "n"(KB), "n"(2 * KB), "n"(3 * KB));
      commit(saddr(&empty[s]));
    }
    commit(saddr(&mma_done));
    if (!ok) *abort = 1;
  }
  __syncwarp();
  // ---- epilogue: every warp, once the last MMA has completed
  {
    const bool got = wait_bounded(saddr(&mma_done), 0, abort);
    mma_ok = __all_sync(0xffffffffu, got) && !*abort;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (mma_ok && u1 > u0) {
    const int C = a.C1 + a.C2;
    for (int t = 0; t < p.tiles; ++t) {
      // warp w reads TMEM lanes 32 w .. 32 w + 31: A rows 128 t + 32 w + lane, row q * SC + ci of
      // input slice q (tap q / Cg, slice cg = q % Cg of the group); rows past the 9 Cg slices are
      // stale operand data and are dropped
      const int row0 = t * 128 + warp * 32;
      if (row0 >= na * SC) break;
      const int q = (row0 + lane) / SC, ci = (row0 + lane) - q * SC;
      const bool valid = q < na;
      const int tap = q / p.Cg, cg = q - tap * p.Cg;
      const int m = tap * C + (grp * p.Cg + cg) * SC + ci;
      for (int n0 = 0; n0 < a.N; n0 += 16) {
        uint32_t r[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * a.N + n0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (!valid) continue;
        float *dst = a.dw + (size_t)m * a.N + n0;
#pragma unroll
        for (int e = 0; e < 16; ++e) atomicAdd(dst + e, __uint_as_float(r[e]));
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0 && abort_sh) atomicExch(err, 1);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

int tmem_cols_of(int n) {
  int c = 32;
  while (c < n) c <<= 1;
  return c;
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// looked up once; the initialisation of a function-local static is thread-safe
EncodeTiled encoder() {
  static const EncodeTiled fn = []() -> EncodeTiled {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiled>(p);
    return nullptr;
  }();
  return fn;
}

}  // namespace

// Forward (bf16 output into a.y) or, with a.dx1 set, a data gradient written as a forward
// convolution of dY (stride 1: with the reversed taps; stride 2: split by output parity, see
// ParityTaps): FP32 into dx1 / dx2.
bool conv_tma_supported(const ConvArgs &a, int mode) {
  const bool out_ok = a.dx1 ? (!a.y && !a.y32 && a.dsplit > 0 && a.dsplit % TM_CH == 0 && a.dsplit <= a.N &&
                               (a.dsplit == a.N || a.dx2))
                            : (a.y && !a.y32);
  return mode == MODE_FWD && a.ks == 3 && (a.stride == 1 || a.stride == 2) && a.pad == 1 && a.C1 > 0 &&
         a.C1 % TM_CH == 0 && a.C2 % TM_CH == 0 && (a.C2 == 0 || a.x2) && out_ok && a.N % 16 == 0 && a.N >= 16 &&
         a.N <= TM_NMAX && a.Nreal <= a.N && encoder() != nullptr;
}

// Forward (bf16 output with bias and ReLU into a.y) or, with a.dx1 set, the data gradient of a 3x3
// stride-1 convolution written as a forward convolution of dY with the reversed taps (FP32 added
// into dx1 / dx2 at the input's pixels; the output grid is the input grid).
bool conv_halo_supported(const ConvArgs &a, int mode) {
  const bool out_ok = a.dx1 ? (!a.y && !a.y32 && a.dsplit > 0 && a.dsplit % TM_CH == 0 && a.dsplit <= a.N &&
                               (a.dsplit == a.N || a.dx2))
                            : (a.y && !a.y32);
  const bool chans = (a.C1 > 0 && a.C1 % TM_CH == 0 && a.C2 % TM_CH == 0 && (a.C2 == 0 || a.x2)) ||
                     (a.C1 == 8 && a.C2 == 0 && !a.dx1);
  return mode == MODE_FWD && a.ks == 3 && a.stride == 1 && a.pad == 1 && chans && out_ok && a.N % 16 == 0 &&
         a.N >= 16 && a.N <= TM_NMAX && a.Nreal <= a.N && (size_t)9 * (a.C1 + a.C2) * a.N * 2 <= HWMAX &&
         encoder() != nullptr;
}

// Tensor maps of the halo variant: the input parts as 4-D (C, W, H, B) bf16 tensors with boxes
// of 8 channels x 10 x 18 pixels x 1 image (16-byte rows, no swizzle, zero fill outside), the
// weight matrix as for the path-2 kernel.
int make_halo_maps(const ConvArgs &a, int Bmax, ConvMaps *m) {
  EncodeTiled enc = encoder();
  if (!enc) return 1;
  std::memset(m, 0, sizeof(*m));
  auto act = [&](CUtensorMap *t, const __nv_bfloat16 *p, int C) {
    const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)a.Win, (cuuint64_t)a.Hin, (cuuint64_t)Bmax};
    const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)a.Win * C * 2, (cuuint64_t)a.Hin * a.Win * C * 2};
    const cuuint32_t box[4] = {8, HW, HH, 1}, es[4] = {1, 1, 1, 1};
    return enc(t, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(p), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  if (!act(&m->x1, a.x1, a.C1)) return 2;
  if (a.C2 > 0 ? !act(&m->x2, a.x2, a.C2) : !act(&m->x2, a.x1, a.C1)) return 3;
  // an 8-channel input: blocks of 8 K values, unswizzled 16-byte rows
  const bool c8 = a.C1 == 8;
  const cuuint64_t wd[2] = {(cuuint64_t)a.K, (cuuint64_t)a.N};
  const cuuint64_t ws[1] = {(cuuint64_t)a.K * 2};
  const cuuint32_t wbox[2] = {c8 ? 8u : (cuuint32_t)TM_CH, (cuuint32_t)a.N}, wes[2] = {1, 1};
  if (enc(&m->w, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(a.w), wd, ws, wbox, wes,
          CU_TENSOR_MAP_INTERLEAVE_NONE, c8 ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_64B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return 4;
  return 0;
}

cudaError_t launch_conv_halo(const ConvArgs &a, const ConvMaps &m, int *err, cudaStream_t st) {
  const int BN = a.N, cols = tmem_cols_of(2 * BN);
  const size_t wbytes = a.C1 == 8 ? (size_t)10 * BN * 16 : (size_t)9 * (a.C1 + a.C2) / TM_CH * BN * 64;
  // the operand windows end inside their stage: the last tap's last core matrix of a plane ends
  // at (2 * 10 + 2) * 16 + 15 * 160 + 128 = 2,880 bytes, the plane's end
  const size_t smem = 1024 + wbytes + (size_t)HSTAGES * HSTAGE;
  cudaError_t e = cudaFuncSetAttribute(k_conv_halo, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_conv_halo, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, smem_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
    return e;
  const int occ = std::max(1, std::min(smem_sm / (int)(smem + 2048), 512 / cols));
  TileGrid tg;
  tg.tx = (a.Wout + HX - 1) / HX;
  tg.ty = (a.Hout + HY - 1) / HY;
  tg.per_img = tg.tx * tg.ty;
  tg.ntiles = tg.per_img * a.Bn;
  const int grid = std::max(1, std::min(tg.ntiles, sms * occ));
  k_conv_halo<<<grid, TM_THREADS, smem, st>>>(m.x1, m.x2, m.w, a, tg, cols, err);
  return cudaGetLastError();
}

// Tensor maps of one convolution: the input parts as 4-D (C, W, H, B) bf16 tensors with boxes
// of 32 channels x 16 x 8 pixels x 1 image (stride s: s * 16 x s * 8 pixels traversed with
// element strides s), the weight matrix [N][K] as a 2-D (K, N) tensor with boxes of 32 x N;
// 64-byte swizzle, zero fill outside.
int make_conv_maps(const ConvArgs &a, int Bmax, ConvMaps *m) {
  EncodeTiled enc = encoder();
  if (!enc) return 1;
  std::memset(m, 0, sizeof(*m));
  auto act = [&](CUtensorMap *t, const __nv_bfloat16 *p, int C) {
    const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)a.Win, (cuuint64_t)a.Hin, (cuuint64_t)Bmax};
    const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)a.Win * C * 2, (cuuint64_t)a.Hin * a.Win * C * 2};
    // a stride-s convolution reads every s-th pixel: a box of s * 16 x s * 8 pixels traversed
    // with element strides s loads the 16 x 8 pixels one tap of an output tile needs
    const cuuint32_t sd = (cuuint32_t)a.stride;
    const cuuint32_t box[4] = {TM_CH, TM_X * sd, TM_Y * sd, 1}, es[4] = {1, sd, sd, 1};
    return enc(t, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(p), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  if (!act(&m->x1, a.x1, a.C1)) return 2;
  if (a.C2 > 0 ? !act(&m->x2, a.x2, a.C2) : !act(&m->x2, a.x1, a.C1)) return 3;
  const cuuint64_t wd[2] = {(cuuint64_t)a.K, (cuuint64_t)a.N};
  const cuuint64_t ws[1] = {(cuuint64_t)a.K * 2};
  const cuuint32_t wbox[2] = {TM_CH, (cuuint32_t)a.N}, wes[2] = {1, 1};
  if (enc(&m->w, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(a.w), wd, ws, wbox, wes,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return 4;
  return 0;
}

namespace {

size_t smem_of(int BN, int S) { return 1024 + (size_t)S * (TM_X * TM_Y * 64 + (size_t)BN * 64); }

// CTAs per SM: as many as the shared memory holds (the ring, the static barriers and the 1 KB
// each CTA reserves) and whose accumulators fit together in the 512 TMEM columns of an SM, so
// that a resident CTA never waits in tcgen05.alloc; a CTA that finds no room starts later.
int occupancy_of(int BN, int S, int cols, int smem_sm) {
  return std::max(1, std::min(smem_sm / (int)(smem_of(BN, S) + 2048), 512 / cols));
}

// Ring depth: 3 stages for N = 32 (6-7 CTAs per SM), 4 for wider layers (their TMEM share caps
// them at 2-4 CTAs per SM); a chain per CTA, so more CTAs per SM beat deeper rings (N = 32: 3
// stages on 7 CTAs within 2 % of 4 on 5, 7 stages on 3 CTAs 12 % slower).  A layer with no more
// tiles than that many resident CTAs takes the deepest ring that still keeps all its tiles
// resident at once (the coarse layers e3a, e3b: 6 stages).  The rate hardly depends on the depth
// (the training step 1 % faster), so load latency does not bound these layers.
int stages_for(int BN, int cols, long ntiles, int sms, int smem_sm) {
  const int S0 = BN <= 32 ? 3 : 4;
  if (ntiles > (long)sms * occupancy_of(BN, S0, cols, smem_sm)) return S0;
  int S = S0;
  while (S < TM_MAXS && ntiles <= (long)sms * occupancy_of(BN, S + 1, cols, smem_sm)) ++S;
  return S;
}

}  // namespace

namespace {

cudaError_t launch_conv_tma_impl(const ConvArgs &a, const ConvMaps &m, const ParityTaps &pt, int *err,
                                 cudaStream_t st) {
  const int BN = a.N, cols = tmem_cols_of(2 * BN);
  int dev = 0, sms = 0, smem_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
    return e;
  TileGrid tg;
  tg.tx = (a.Wout + TM_X - 1) / TM_X;
  tg.ty = (a.Hout + TM_Y - 1) / TM_Y;
  tg.per_img = tg.tx * tg.ty;
  tg.ntiles = tg.per_img * a.Bn;
  ParityTaps p = pt;
  if (p.on) {
    p.per_class = tg.ntiles;
    tg.ntiles *= 4;
  }
  const int S = stages_for(BN, cols, tg.ntiles, sms, smem_sm);
  const size_t smem = smem_of(BN, S);
  const int occ = occupancy_of(BN, S, cols, smem_sm);
  e = cudaFuncSetAttribute(k_conv_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_conv_tma, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, std::min(tg.ntiles, sms * occ));
  k_conv_tma<<<grid, TM_THREADS, smem, st>>>(m.x1, m.x2, m.w, a, tg, p, S, cols, err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_conv_tma(const ConvArgs &a, const ConvMaps &m, int *err, cudaStream_t st) {
  ParityTaps off;
  std::memset(&off, 0, sizeof(off));
  return launch_conv_tma_impl(a, m, off, err, st);
}

// Data gradient of a stride-2 3x3 layer on the coarse grid of dY (a: a stride-1 convolution of dY,
// a.x1 = dY with C1 = its channels, Hout x Wout = dY's grid, a.w = wd, the data-gradient weights
// with the taps in their own order, the FP32 data-gradient outputs), written on the Hf x Wf input
// grid by output parity.
cudaError_t launch_conv_tma_parity(const ConvArgs &a, const ConvMaps &m, int Hf, int Wf, int *err, cudaStream_t st) {
  ParityTaps p;
  std::memset(&p, 0, sizeof(p));
  p.on = 1;
  p.Hf = Hf;
  p.Wf = Wf;
  for (int pa = 0; pa < 2; ++pa)
    for (int pc = 0; pc < 2; ++pc) {
      const int cls = 2 * pa + pc;
      int n = 0;
      for (int kh = 0; kh < 3; ++kh)
        for (int kw = 0; kw < 3; ++kw) {
          if ((kh + pa + 1) % 2 || (kw + pc + 1) % 2) continue;  // kh = a + 1, kw = c + 1 (mod 2)
          p.dy[cls][n] = (pa + 1 - kh) / 2;
          p.dx[cls][n] = (pc + 1 - kw) / 2;
          p.tap[cls][n] = 3 * kh + kw;
          ++n;
        }
      p.n[cls] = n;
    }
  return launch_conv_tma_impl(a, m, p, err, st);
}

namespace {

// Plan: the input slice width (32 channels; 8 for an input of 8 channels), the channel group Cg
// (a divisor of the input's slices whose accumulator tiles fit in the 512 TMEM columns) and the
// segment of 64 or 128 pixels whose stage fits at least twice in shared memory, chosen by a model
// of the load side, which sets the pace (measured: a TMA box costs about 100 SM cycles plus one
// per line it brings): groups x boxes x (100 + pixels) / pixels per output pixel, padding
// included.  The segment shape P x R: the one with the fewest padded pixels.
constexpr size_t WT_SMEM_MAX = 225 * 1024;

int wgrad_slice_channels(const ConvArgs &a) {
  if (a.C1 % 32 == 0 && a.C2 % 32 == 0) return 32;
  if (a.C1 == 8 && a.C2 == 0) return 8;
  return 0;
}

void wgrad_stage(const WgPlan &p, size_t *stage, size_t *guard) {
  *stage = (size_t)p.a_slots * p.slice + (size_t)p.nb * p.bslice;
  // a last tile reads 128 / sc slices from its first: past the stage's end by at most this much
  const size_t reach = (size_t)p.tiles * (128 / p.sc) * p.slice;
  *guard = reach > *stage ? reach - *stage : 0;
}

WgPlan wgrad_plan(const ConvArgs &a) {
  WgPlan p;
  std::memset(&p, 0, sizeof(p));
  p.sc = wgrad_slice_channels(a);
  if (p.sc == 0) return p;
  const int spt = 128 / p.sc;
  p.c1 = a.C1 / p.sc;
  const int cs = (a.C1 + a.C2) / p.sc;
  p.nb = a.N / 32;
  double best_cost = 0.0;
  for (int cg = cs; cg >= 1; --cg) {
    if (cs % cg) continue;
    const int tiles = (9 * cg + spt - 1) / spt;
    if (tiles * a.N > 512) continue;
    for (int pix = 64; pix <= 128; pix *= 2) {
      WgPlan q = p;
      q.Cg = cg;
      q.tiles = tiles;
      q.pix = pix;
      q.slice = (uint32_t)(pix * p.sc * 2);
      q.bslice = (uint32_t)(pix * 64);
      q.a_slots = p.sc == 32 ? 9 * cg : tiles * spt;
      size_t stage, guard;
      wgrad_stage(q, &stage, &guard);
      q.S = (int)std::min<size_t>(WT_MAXS, (WT_SMEM_MAX - 1024 - guard) / stage);
      if (q.S < 2) continue;
      long padded = -1;  // output pixels of the best segment shape, padding included
      for (int P = 8; P <= pix; P *= 2) {
        const int R = pix / P;
        const long n = (long)((a.Wout + P - 1) / P) * P * (long)((a.Hout + R - 1) / R) * R;
        if (padded < 0 || n < padded) padded = n;
      }
      const double cost = (double)(cs / cg) * (9 * cg + p.nb) * (100.0 + pix) / pix * (double)padded;
      if (p.Cg == 0 || cost < best_cost) {
        best_cost = cost;
        p = q;
      }
    }
  }
  if (p.Cg == 0) return p;
  long best = -1;
  for (int P = 8; P <= p.pix; P *= 2) {
    const int R = p.pix / P;
    const long padded = (long)((a.Wout + P - 1) / P) * P * (long)((a.Hout + R - 1) / R) * R;
    if (best < 0 || padded < best) best = padded, p.P = P, p.R = R;
  }
  p.tx = (a.Wout + p.P - 1) / p.P;
  p.per_img = p.tx * ((a.Hout + p.R - 1) / p.R);
  p.units = p.per_img * a.Bn;
  return p;
}

size_t wgrad_smem(const WgPlan &p) {
  size_t stage, guard;
  wgrad_stage(p, &stage, &guard);
  return 1024 + (size_t)p.S * stage + guard;
}

}  // namespace

bool wgrad_tma_supported(const ConvArgs &a) {
  if (!(a.ks == 3 && (a.stride == 1 || a.stride == 2) && a.pad == 1 && a.C1 > 0 && (a.C2 == 0 || a.x2) &&
        a.N % 32 == 0 && a.N >= 32 && a.N <= 128 && a.Cout == a.N && a.M == a.Kf && a.Pout > 0 &&
        encoder() != nullptr))
    return false;
  return wgrad_plan(a).Cg > 0;
}

// Tensor maps of the weight gradient: the input parts as 4-D (C, W, H, B) tensors with boxes of
// sc channels x sP x sR pixels traversed with element strides s (the stride; 64-byte swizzle for
// 32-channel slices, none for 8), dY as a 4-D (N, Wout, Hout, B) tensor with boxes of 32 x P x R
// (64-byte swizzle); zero fill outside.  The dY map goes into the w slot of ConvMaps.
int make_wgrad_maps(const ConvArgs &a, int Bmax, ConvMaps *m) {
  EncodeTiled enc = encoder();
  if (!enc) return 1;
  const WgPlan p = wgrad_plan(a);
  if (p.Cg == 0) return 5;
  std::memset(m, 0, sizeof(*m));
  const cuuint32_t sd = (cuuint32_t)a.stride;
  auto map4 = [&](CUtensorMap *t, const __nv_bfloat16 *ptr, int C, int W, int H, cuuint32_t s, int box_c) {
    const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)Bmax};
    const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
    const cuuint32_t box[4] = {(cuuint32_t)box_c, (cuuint32_t)p.P * s, (cuuint32_t)p.R * s, 1}, es[4] = {1, s, s, 1};
    return enc(t, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(ptr), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, box_c == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  if (!map4(&m->x1, a.x1, a.C1, a.Win, a.Hin, sd, p.sc)) return 2;
  if (a.C2 > 0 ? !map4(&m->x2, a.x2, a.C2, a.Win, a.Hin, sd, p.sc) : !map4(&m->x2, a.x1, a.C1, a.Win, a.Hin, sd, p.sc))
    return 3;
  if (!map4(&m->w, a.dy, a.N, a.Wout, a.Hout, 1, 32)) return 4;
  return 0;
}

cudaError_t launch_wgrad_tma(const ConvArgs &a, const ConvMaps &m, int *err, cudaStream_t st) {
  WgPlan p = wgrad_plan(a);
  if (p.Cg <= 0) return cudaErrorInvalidValue;
  const int cols = tmem_cols_of(p.tiles * a.N);
  const size_t smem = wgrad_smem(p);
  auto kern = p.sc == 32 ? k_wgrad_tma<32> : k_wgrad_tma<8>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, smem_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
    return e;
  const int occ = std::max(1, std::min(smem_sm / (int)(smem + 2048), 512 / cols));
  const int groups = (a.C1 + a.C2) / p.sc / p.Cg;
  // pixel ranges: fill the GPU once, but give every CTA at least 16 segments (each CTA ends
  // with one FP32 atomic per weight of its group)
  const int splits = std::max(1, std::min((sms * occ + groups - 1) / groups, (p.units + 15) / 16));
  p.per_cta = (p.units + splits - 1) / splits;
  const int gx = (p.units + p.per_cta - 1) / p.per_cta;
  kern<<<dim3(gx, groups), WT_THREADS, smem, st>>>(m.x1, m.x2, m.w, a, p, cols, err);
  return cudaGetLastError();
}

}  // namespace unk
