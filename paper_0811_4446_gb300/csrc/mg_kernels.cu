// CUDA kernels of the axisymmetric drift-diffusion / Poisson multigrid solver (FP64 path).
//
// Paper: Ristivojevic & Petrovic, arXiv:0811.4446, Sec. 2.
//  * coefficient build: Scharfetter-Gummel face fluxes (eqs. 8-11) and their
//    derivatives, which make up the 3x3 blocks of the Newton system (eq. 14);
//  * nonlinear residual: eq. 7 for both species and eqs. 12-13 (Poisson), in
//    finite-volume form (rows multiplied by the control volume);
//  * red-black collective (3x3 point-block) Gauss-Seidel smoother, linear
//    residual, full-weighting restriction R = P^T, bilinear prolongation, dense
//    coarsest-level inverse: the multigrid solver of eq. 14.
//
// Thread mapping: one thread per node (or per node of one colour), 32 x 8 blocks,
// x = radial index (coalesced), y = axial index.
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include <cstdio>

#include "mg_impl.cuh"

namespace mgk {

static unsigned long long g_launches = 0;
static thread_local bool g_capturing = false;
static thread_local int g_captured = 0;
void set_capturing(bool on) { g_capturing = on; g_captured = 0; }
int captured_launches() { return g_captured; }
void count_launch(int n) {
  if (g_capturing) g_captured += n;
  else __atomic_add_fetch(&g_launches, (unsigned long long)n, __ATOMIC_RELAXED);
}
unsigned long long total_launches() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

constexpr int BX = 32, BY = 8, NT = BX * BY;

// ---- programmatic dependent launch ----------------------------------------------------------
// A kernel launched with programmatic stream serialization may start while the kernel before it
// in the stream is still running, once every CTA of that kernel has executed
// griddepcontrol.launch_dependents; griddepcontrol.wait then blocks until the previous kernel
// has completed and its memory is visible.  The V-cycle kernels signal their dependents at once
// and read only data that no kernel of the linear solve writes (face coefficients, factors,
// conductances) before they wait.  Without the launch attribute both instructions are no-ops.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_k(bool pdl, void (*kern)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t st, Args... args) {
  if (!pdl) {
    kern<<<g, b, smem, st>>>(args...);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// ------------------------------------------------------------------------------------------
// Bernoulli function B(x) = x / (e^x - 1): F(x) = B(x), G(x) = B(-x) (definitions after eq. 11).
// Returns B(x), B(-x), B'(x), B'(-x).  |x| < 0.1: Bernoulli-number series
// (B_2 = 1/6, B_4 = -1/30, B_6 = 1/42, B_8 = -1/30, B_10 = 5/66); otherwise, for y = |x|,
// B(y) = y e^{-y} / (1 - e^{-y}) with 1 - e^{-y} = -expm1(-y) (no overflow), and the
// reflections B(-y) = B(y) + y, B'(-y) = -B'(y) - 1.
struct Bern {
  double Bp, Bm, dBp, dBm;
};

__device__ __forceinline__ Bern bernoulli(double x) {
  const double y = fabs(x);
  double by, dby;
  if (y < 0.1) {
    const double y2 = y * y;
    const double even =
        1.0 + y2 * (1.0 / 12.0 +
                    y2 * (-1.0 / 720.0 + y2 * (1.0 / 30240.0 + y2 * (-1.0 / 1209600.0 + y2 * (1.0 / 47900160.0)))));
    by = even - 0.5 * y;
    const double odd =
        y * (1.0 / 6.0 + y2 * (-1.0 / 180.0 + y2 * (1.0 / 5040.0 + y2 * (-1.0 / 151200.0 + y2 * (1.0 / 4790016.0)))));
    dby = odd - 0.5;
  } else {
    const double t = exp(-y);
    const double em = -expm1(-y);
    by = y * t / em;
    dby = t * (em - y) / (em * em);
  }
  Bern b;
  if (x >= 0.0) {
    b.Bp = by; b.Bm = by + y; b.dBp = dby; b.dBm = -dby - 1.0;
  } else {
    b.Bp = by + y; b.Bm = by; b.dBp = -dby - 1.0; b.dBm = dby;
  }
  return b;
}

// ------------------------------------------------------------------------------------------
// Transport at a face: constants, or linear interpolation in |E| between table rows.
struct FaceTr {
  double mu_e, D_e, mu_p, D_p;
};

__device__ __forceinline__ FaceTr lookup(const Transport &tr, double Eabs) {
  const double *T = tr.table;
  const int n = tr.rows;
  const double x = fmin(fmax(Eabs, __ldg(T)), __ldg(T + 5 * (n - 1)));
  int lo = 0, hi = n - 1;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(T + 5 * mid) <= x) lo = mid; else hi = mid;
  }
  const double *a = T + 5 * lo, *b = a + 5;
  const double t = (x - __ldg(a)) / (__ldg(b) - __ldg(a));
  FaceTr f;
  f.mu_e = (__ldg(a + 1) + t * (__ldg(b + 1) - __ldg(a + 1))) * tr.inv_pf;
  f.D_e = (__ldg(a + 2) + t * (__ldg(b + 2) - __ldg(a + 2))) * tr.inv_pf;
  f.mu_p = (__ldg(a + 3) + t * (__ldg(b + 3) - __ldg(a + 3))) * tr.inv_pf;
  f.D_p = (__ldg(a + 4) + t * (__ldg(b + 4) - __ldg(a + 4))) * tr.inv_pf;
  return f;
}

// |E| on the r-face (i+1/2, j) (1 <= j <= nz-1): normal part across the face, transverse part the
// mean of the four adjacent z-face fields (E = -grad V, eq. 6).
__device__ __forceinline__ double eabs_rface(const Level &L, const double *V, int j, int i) {
  const size_t k = (size_t)j * L.P + i;
  const double En = -(V[k + 1] - V[k]) / L.dr;
  const double dzm = L.dz[j - 1], dzp = L.dz[j];
  const double a = -(V[k] - V[k - L.P]) / dzm, b = -(V[k + L.P] - V[k]) / dzp;
  const double c = -(V[k + 1] - V[k + 1 - L.P]) / dzm, d = -(V[k + 1 + L.P] - V[k + 1]) / dzp;
  const double Et = 0.25 * (((a + b) + c) + d);
  return sqrt(En * En + Et * Et);
}

// |E| on the z-face (i, j+1/2) (0 <= j <= nz-1): the transverse part is zero on the axis and
// on the outer wall (dV/dr = 0 there by symmetry).
__device__ __forceinline__ double eabs_zface(const Level &L, const double *V, int j, int i) {
  const size_t k = (size_t)j * L.P + i;
  const double En = -(V[k + L.P] - V[k]) / L.dz[j];
  double Et = 0.0;
  if (i > 0 && i < L.nr) {
    const double a = -(V[k] - V[k - 1]) / L.dr, b = -(V[k + 1] - V[k]) / L.dr;
    const double c = -(V[k + L.P] - V[k + L.P - 1]) / L.dr, d = -(V[k + L.P + 1] - V[k + L.P]) / L.dr;
    Et = 0.25 * (((a + b) + c) + d);
  }
  return sqrt(En * En + Et * Et);
}

__device__ __forceinline__ FaceTr tr_rface(const Level &L, const Transport &tr, const double *V, int j, int i) {
  if (!tr.table) return FaceTr{tr.mu_e, tr.D_e, tr.mu_p, tr.D_p};
  return lookup(tr, eabs_rface(L, V, j, i));
}
__device__ __forceinline__ FaceTr tr_zface(const Level &L, const Transport &tr, const double *V, int j, int i) {
  if (!tr.table) return FaceTr{tr.mu_e, tr.D_e, tr.mu_p, tr.D_p};
  return lookup(tr, eabs_zface(L, V, j, i));
}

// ---- coefficient path with few FP64 divisions and transcendentals -----------------------------
// FP64 arithmetic is the scarce resource of the face evaluation (the FP64 pipe issues one warp
// instruction per SM sub-partition every 64 cycles on this part): the faces below use stored
// reciprocals of the spacings and table intervals, and one exponential and one division per
// Bernoulli pair.  For y = |x| >= 0.1: e = 1 - e^{-y} from expm1 when y < 0.5 (then e^{-y} =
// 1 - e > 0.6 is exact to an ulp) and from exp otherwise (then e > 0.39 is), so both keep full
// relative accuracy; B(y) = y e^{-y} / e, B'(y) = e^{-y} (e - y) / e^2.
__device__ __forceinline__ Bern bernoulli1(double x) {
  const double y = fabs(x);
  double by, dby;
  if (y < 0.1) {
    const double y2 = y * y;
    const double even =
        1.0 + y2 * (1.0 / 12.0 +
                    y2 * (-1.0 / 720.0 + y2 * (1.0 / 30240.0 + y2 * (-1.0 / 1209600.0 + y2 * (1.0 / 47900160.0)))));
    by = even - 0.5 * y;
    const double odd =
        y * (1.0 / 6.0 + y2 * (-1.0 / 180.0 + y2 * (1.0 / 5040.0 + y2 * (-1.0 / 151200.0 + y2 * (1.0 / 4790016.0)))));
    dby = odd - 0.5;
  } else {
    double t, em;
    if (y < 0.5) { em = -expm1(-y); t = 1.0 - em; }
    else { t = exp(-y); em = 1.0 - t; }
    const double ie = 1.0 / em;
    const double tie = t * ie;
    by = y * tie;
    dby = tie * (em - y) * ie;
  }
  Bern b;
  if (x >= 0.0) {
    b.Bp = by; b.Bm = by + y; b.dBp = dby; b.dBm = -dby - 1.0;
  } else {
    b.Bp = by + y; b.Bm = by; b.dBp = -dby - 1.0; b.dBm = dby;
  }
  return b;
}

__device__ __forceinline__ FaceTr lookup1(const Transport &tr, double Eabs) {
  const double *T = tr.table;
  const int n = tr.rows;
  const double x = fmin(fmax(Eabs, __ldg(T)), __ldg(T + 5 * (n - 1)));
  int lo = 0, hi = n - 1;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(T + 5 * mid) <= x) lo = mid; else hi = mid;
  }
  const double *a = T + 5 * lo, *b = a + 5;
  const double t = (x - __ldg(a)) * __ldg(tr.inv_dE + lo);
  FaceTr f;
  f.mu_e = (__ldg(a + 1) + t * (__ldg(b + 1) - __ldg(a + 1))) * tr.inv_pf;
  f.D_e = (__ldg(a + 2) + t * (__ldg(b + 2) - __ldg(a + 2))) * tr.inv_pf;
  f.mu_p = (__ldg(a + 3) + t * (__ldg(b + 3) - __ldg(a + 3))) * tr.inv_pf;
  f.D_p = (__ldg(a + 4) + t * (__ldg(b + 4) - __ldg(a + 4))) * tr.inv_pf;
  return f;
}

// |E| on the r-face (i+1/2, j) and the z-face (i, j+1/2), as eabs_rface / eabs_zface.
__device__ __forceinline__ double eabs_r1(const Level &L, const double *V, int j, size_t k) {
  const int P = L.P;
  const double En = (V[k] - V[k + 1]) * L.idr;
  const double lo = (V[k - P] - V[k]) + (V[k + 1 - P] - V[k + 1]);
  const double up = (V[k] - V[k + P]) + (V[k + 1] - V[k + 1 + P]);
  const double Et = 0.25 * (lo * L.idz[j - 1] + up * L.idz[j]);
  return sqrt(En * En + Et * Et);
}
__device__ __forceinline__ double eabs_z1(const Level &L, const double *V, int j, int i, size_t k) {
  const int P = L.P;
  const double En = (V[k] - V[k + P]) * L.idz[j];
  double Et = 0.0;
  if (i > 0 && i < L.nr)
    Et = 0.25 * L.idr * ((V[k - 1] - V[k + 1]) + (V[k + P - 1] - V[k + P + 1]));
  return sqrt(En * En + Et * Et);
}

// Face coefficients (cG, cF, cV) of both species on one face.
__device__ __forceinline__ void face_coefs(const Transport &tr, bool table, double Eabs, double g, double dV,
                                           double neL, double neR, double npL, double npR, double (&c)[NCOEF]) {
  const FaceTr t = table ? lookup1(tr, Eabs) : FaceTr{tr.mu_e, tr.D_e, tr.mu_p, tr.D_p};
  {
    const Bern b = bernoulli1((t.mu_e / t.D_e) * dV);  // electrons: s = -1
    const double gD = g * t.D_e;
    c[CGE] = gD * b.Bm; c[CFE] = gD * b.Bp;
    c[CVE] = -g * t.mu_e * (neL * b.dBm + neR * b.dBp);
  }
  {
    const Bern b = bernoulli1(-(t.mu_p / t.D_p) * dV);  // ions: s = +1
    const double gD = g * t.D_p;
    c[CGP] = gD * b.Bm; c[CFP] = gD * b.Bp;
    c[CVP] = g * t.mu_p * (npL * b.dBm + npR * b.dBp);
  }
}

// East r-face and north z-face coefficients of node (i, j) of level L (face conductances g:
// the stored Poisson ones, (i + 1/2) dz_c and vol_r / dz).
__device__ __forceinline__ void coef_node(const Level &L, const StateView &sv, const Transport &tr, int i, int j) {
  const size_t k = (size_t)j * L.P + i;
  const double *ne = sv.u[NE], *np = sv.u[NP], *V = sv.u[NV];
  const bool table = tr.table != nullptr;
  double c[NCOEF];
  if (i < L.nr && j >= 1 && j < L.nz) {
    face_coefs(tr, table, table ? eabs_r1(L, V, j, k) : 0.0, L.gR[k], V[k + 1] - V[k], ne[k], ne[k + 1], np[k],
               np[k + 1], c);
#pragma unroll
    for (int a = 0; a < NCOEF; ++a) L.cr[a][k] = c[a];
  }
  if (j < L.nz) {
    face_coefs(tr, table, table ? eabs_z1(L, V, j, i, k) : 0.0, L.gZ[k], V[k + L.P] - V[k], ne[k], ne[k + L.P],
               np[k], np[k + L.P], c);
#pragma unroll
    for (int a = 0; a < NCOEF; ++a) L.cz[a][k] = c[a];
  }
}

// SG flux through a face from L to R (eqs. 8-11): alpha = -s (mu/D)(V_R - V_L),
// flux = g D (n_L G(alpha) - n_R F(alpha)).
__device__ __forceinline__ double sg_flux(double g, double mu, double D, double s, double nL, double nR,
                                          double dV) {
  const Bern b = bernoulli(-s * (mu / D) * dV);
  return g * D * (nL * b.Bm - nR * b.Bp);
}

// Derivatives of the SG flux: cG = d/dn_L, cF = -d/dn_R, cV = d/dV_R = -d/dV_L (mu, D frozen).
__device__ __forceinline__ void sg_coef(double g, double mu, double D, double s, double nL, double nR, double dV,
                                        double &cG, double &cF, double &cV) {
  const Bern b = bernoulli(-s * (mu / D) * dV);
  cG = g * D * b.Bm;
  cF = g * D * b.Bp;
  // G'(a) = -B'(-a), F'(a) = B'(a):  cV = -s g mu (n_L G' - n_R F') = s g mu (n_L B'(-a) + n_R B'(a))
  cV = s * g * mu * (nL * b.dBm + nR * b.dBp);
}

// ------------------------------------------------------------------------------------------
// Deterministic block reduction: every block writes K partials, the last block to finish sums
// them in block order and writes out[K].  op: 0 = sum, 1 = max.
template <int K>
__device__ void reduce_finish(double (&v)[K], double *partials, unsigned *counter, double *out, int op) {
  __shared__ double sh[K][NT / 32];
  __shared__ bool last;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    double x = v[q];
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_down_sync(0xffffffffu, x, o);
      x = op ? fmax(x, y) : x + y;
    }
    if (lane == 0) sh[q][wid] = x;
  }
  __syncthreads();
  const int nblocks = gridDim.x * gridDim.y;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      double x = sh[q][0];
      for (int w = 1; w < nwarps; ++w) x = op ? fmax(x, sh[q][w]) : x + sh[q][w];
      partials[(size_t)bid * K + q] = x;
    }
    __threadfence();
    const unsigned done = atomicAdd(counter, 1u);
    last = (done == (unsigned)nblocks - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int nthr = blockDim.x * blockDim.y;
  // each thread folds blocks tid, tid + nthr, ... in that order, four blocks' partials per
  // round with all their loads in flight (L2 reads, .cg: the other blocks' writes are visible
  // after their fence and the counter); a dependent load per block made this pass the longest
  // part of a norm launch
  double xs[K];
  bool first = true;
#pragma unroll
  for (int q = 0; q < K; ++q) xs[q] = 0.0;
  int b = tid;
  for (; b + 3 * nthr < nblocks; b += 4 * nthr) {
    double y[4][K];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int q = 0; q < K; ++q) y[u][q] = __ldcg(partials + (size_t)(b + u * nthr) * K + q);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int q = 0; q < K; ++q)
        xs[q] = (first && u == 0) ? y[u][q] : (op ? fmax(xs[q], y[u][q]) : xs[q] + y[u][q]);
    first = false;
  }
  for (; b < nblocks; b += nthr) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const double y = __ldcg(partials + (size_t)b * K + q);
      xs[q] = first ? y : (op ? fmax(xs[q], y) : xs[q] + y);
    }
    first = false;
  }
#pragma unroll
  for (int q = 0; q < K; ++q) {
    double x = first ? (op ? -1.0 : 0.0) : xs[q];
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_down_sync(0xffffffffu, x, o);
      x = op ? fmax(x, y) : x + y;
    }
    if (lane == 0) sh[q][wid] = x;
  }
  __syncthreads();
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      double x = sh[q][0];
      for (int w = 1; w < nwarps; ++w) x = op ? fmax(x, sh[q][w]) : x + sh[q][w];
      out[q] = x;
    }
    *counter = 0u;
  }
}

// ------------------------------------------------------------------------------------------
// K1: face coefficients (eqs. 8-11 differentiated) for the east r-face and north z-face of each node.
constexpr int CBY = 2;  // 32 x 2 threads: the FP64-bound set-up kernels spread over every SM

__global__ void __launch_bounds__(32 * CBY) k_coef(Level L, StateView sv, Transport tr) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * CBY + threadIdx.y;
  if (i > L.nr || j > L.nz) return;
  coef_node(L, sv, tr, i, j);
}

cudaError_t launch_coef(const Level &L, const StateView &sv, const Transport &tr, cudaStream_t st) {
  dim3 b(32, CBY), g((L.nr + 1 + 31) / 32, (L.nz + 1 + CBY - 1) / CBY);
  k_coef<<<g, b, 0, st>>>(L, sv, tr);
  count_launch();
  return cudaGetLastError();
}

// All levels a .. b in one launch (grid sized by level a, the largest).
__global__ void __launch_bounds__(32 * CBY) k_coef_levels(const LevelSet *__restrict__ S, int a, Transport tr) {
  const int l = a + blockIdx.z;
  const Level &L = S->L[l];
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * CBY + threadIdx.y;
  if (i > L.nr || j > L.nz) return;
  coef_node(L, S->sv[l], tr, i, j);
}

cudaError_t launch_coef_levels(const LevelSet *S, const Level &La, int a, int b, const Transport &tr,
                               cudaStream_t st) {
  if (b < a) return cudaSuccess;
  dim3 bl(32, CBY), g((La.nr + 1 + 31) / 32, (La.nz + 1 + CBY - 1) / CBY, b - a + 1);
  k_coef_levels<<<g, bl, 0, st>>>(S, a, tr);
  count_launch();
  return cudaGetLastError();
}

// Injection of the state of level l0 into levels l0 + 1 .. l1 (node (I, J) of level l is node
// (I, J) x 2^(l - l0) of level l0 on the nested grids).
__global__ void k_inject_levels(const LevelSet *__restrict__ S, int l0) {
  const int l = l0 + 1 + blockIdx.z;
  const Level &C = S->L[l];
  const int I = blockIdx.x * 32 + threadIdx.x;
  const int J = blockIdx.y * CBY + threadIdx.y;
  if (I > C.nr || J > C.nz) return;
  const int sh = l - l0;
  const size_t kc = (size_t)J * C.P + I, kf = ((size_t)J << sh) * S->L[l0].P + ((size_t)I << sh);
#pragma unroll
  for (int q = 0; q < 3; ++q) S->sv[l].u[q][kc] = S->sv[l0].u[q][kf];
}

cudaError_t launch_inject_levels(const LevelSet *S, const Level &L0, int l0, int l1, cudaStream_t st) {
  if (l1 <= l0) return cudaSuccess;
  const int nr = L0.nr / 2, nz = L0.nz / 2;
  dim3 bl(32, CBY), g((nr + 1 + 31) / 32, (nz + 1 + CBY - 1) / CBY, l1 - l0);
  k_inject_levels<<<g, bl, 0, st>>>(S, l0);
  count_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// K2': nonlinear residual from the face coefficients of the same state: the SG flux through a
// face is cG n_L - cF n_R (cG = g D G(alpha), cF = g D F(alpha)), the Poisson flux g dV.
// The steady rows (sources, fluxes, space charge) are summed first and the time-derivative
// terms added last, so with steady_too the same launch also reduces the steady rows' sums
// (into out[6..11]), equal bit for bit to a launch with dt_inv = 0, writes -F of the steady
// rows (colour-split) into fs, and reduces sum(Ts t) and sum(t^2) of both continuity rows
// (out[12..15]), t = A (|n| + |n|): the residual of a step that starts from this state (u_old
// = u, so the time term of F vanishes) has the steady F, and its term norms follow for any dt
// from sum((Ts + t / dt)^2) = sum(Ts^2) + 2 sum(Ts t) / dt + sum(t^2) / dt^2.
// One unknown row of k_resid_coef: F and T of node (i, j), the 16 sums' terms in acc (zero
// outside the unknown rows), f / F / fs written as requested.
__device__ __forceinline__ void resid_row(const Level &L, const StateView &sv, double dt_inv, int write_f,
                                          int steady_too, double *F0, double *F1, double *F2, double *fs0,
                                          double *fs1, double *fs2, int i, int j, double (&acc)[16]) {
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.0;
  if (i < L.ni && j < L.nz) {
    const int P = L.P;
    const size_t k = (size_t)j * P + i;
    const double *ne = sv.u[NE], *np = sv.u[NP], *V = sv.u[NV];
    const double A = L.volr[i] * L.dzc[j];
    double Fe = 0, Fp = 0, FV = 0, Te = 0, Tp = 0, TV = 0;
    Fe -= A * sv.S[0][k];
    Fp -= A * sv.S[1][k];
    Te += A * fabs(sv.S[0][k]);
    Tp += A * fabs(sv.S[1][k]);
    auto face = [&](double *const *c, const double *gp, size_t kL, size_t kR, size_t kc, double sgn) {
      const double pe = c[CGE][kc] * ne[kL] - c[CFE][kc] * ne[kR];
      const double pp = c[CGP][kc] * np[kL] - c[CFP][kc] * np[kR];
      const double ps = gp[kc] * (V[kR] - V[kL]);
      Fe += sgn * pe; Fp += sgn * pp; FV += sgn * ps;
      Te += fabs(pe); Tp += fabs(pp); TV += fabs(ps);
    };
    if (i < L.nr) face(L.cr, L.gR, k, k + 1, k, 1.0);
    if (i > 0) face(L.cr, L.gR, k - 1, k, k - 1, -1.0);
    face(L.cz, L.gZ, k, k + P, k, 1.0);
    face(L.cz, L.gZ, k - P, k, k - P, -1.0);
    const double ak = L.Ak[k];
    FV += ak * (np[k] - ne[k]);
    TV += ak * (fabs(np[k]) + fabs(ne[k]));
    acc[6] = Fe * Fe; acc[7] = Fp * Fp; acc[8] = FV * FV;
    acc[9] = Te * Te; acc[10] = Tp * Tp; acc[11] = TV * TV;
    if (steady_too) {
      const double te = A * (fabs(ne[k]) + fabs(ne[k])), tp = A * (fabs(np[k]) + fabs(np[k]));
      acc[12] = Te * te; acc[13] = te * te; acc[14] = Tp * tp; acc[15] = tp * tp;
      if (fs0) {
        const size_t kf = cidx(P, i, j);
        fs0[kf] = -Fe; fs1[kf] = -Fp; fs2[kf] = -FV;
      }
    }
    if (dt_inv > 0.0) {
      Fe += A * (ne[k] - sv.uold[NE][k]) * dt_inv;
      Fp += A * (np[k] - sv.uold[NP][k]) * dt_inv;
      Te += A * (fabs(ne[k]) + fabs(sv.uold[NE][k])) * dt_inv;
      Tp += A * (fabs(np[k]) + fabs(sv.uold[NP][k])) * dt_inv;
    }
    if (write_f) {
      const size_t kf = cidx(P, i, j);
      L.f[NE][kf] = -Fe; L.f[NP][kf] = -Fp; L.f[NV][kf] = -FV;
    }
    if (F0) { F0[k] = Fe; F1[k] = Fp; F2[k] = FV; }
    acc[0] = Fe * Fe; acc[1] = Fp * Fp; acc[2] = FV * FV;
    acc[3] = Te * Te; acc[4] = Tp * Tp; acc[5] = TV * TV;
  }
}

__global__ void __launch_bounds__(32 * CBY) k_resid_coef(Level L, StateView sv, double dt_inv, int write_f,
                                                         int steady_too, double *F0, double *F1, double *F2,
                                                         double *fs0, double *fs1, double *fs2, double *partials,
                                                         unsigned *counter, double *out) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * CBY + threadIdx.y + 1;
  double acc[16];
  resid_row(L, sv, dt_inv, write_f, steady_too, F0, F1, F2, fs0, fs1, fs2, i, j, acc);
  if (steady_too) {
    reduce_finish<16>(acc, partials, counter, out, 0);
  } else {
    double a6[6] = {acc[0], acc[1], acc[2], acc[3], acc[4], acc[5]};
    reduce_finish<6>(a6, partials, counter, out, 0);
  }
}

cudaError_t launch_resid_coef(const Level &L, const StateView &sv, double dt, bool write_f, bool steady_too,
                              double *Fout[3], double *const fsteady[3], double *partials, unsigned *counter,
                              double *out, cudaStream_t st) {
  dim3 b(32, CBY), g((L.nr + 1 + 31) / 32, (L.nz - 1 + CBY - 1) / CBY);
  k_resid_coef<<<g, b, 0, st>>>(L, sv, dt > 0 ? 1.0 / dt : 0.0, write_f ? 1 : 0, steady_too ? 1 : 0,
                                Fout ? Fout[0] : nullptr, Fout ? Fout[1] : nullptr, Fout ? Fout[2] : nullptr,
                                fsteady ? fsteady[0] : nullptr, fsteady ? fsteady[1] : nullptr,
                                fsteady ? fsteady[2] : nullptr, partials, counter, out);
  count_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// K2: nonlinear residual (eq. 7 x control volume; eqs. 12-13 x control volume) and term sums.
__global__ void k_residual(Level L, StateView sv, Transport tr, double dt_inv, int write_f, double *F0,
                           double *F1, double *F2, double *partials, unsigned *counter, double *out6) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y + 1;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  if (i <= L.nr && j < L.nz) {
    const int P = L.P;
    const size_t k = (size_t)j * P + i;
    const double *ne = sv.u[NE], *np = sv.u[NP], *V = sv.u[NV];
    const double A = L.volr[i] * L.dzc[j];
    double Fe = 0, Fp = 0, FV = 0, Te = 0, Tp = 0, TV = 0;
    if (dt_inv > 0.0) {
      Fe += A * (ne[k] - sv.uold[NE][k]) * dt_inv;
      Fp += A * (np[k] - sv.uold[NP][k]) * dt_inv;
      Te += A * (fabs(ne[k]) + fabs(sv.uold[NE][k])) * dt_inv;
      Tp += A * (fabs(np[k]) + fabs(sv.uold[NP][k])) * dt_inv;
    }
    Fe -= A * sv.S[0][k];
    Fp -= A * sv.S[1][k];
    Te += A * fabs(sv.S[0][k]);
    Tp += A * fabs(sv.S[1][k]);
    // faces: sign +1 where this node is the L end (east, north), -1 where it is the R end (west, south)
#pragma unroll
    for (int face = 0; face < 4; ++face) {
      size_t kL, kR;
      double g;
      FaceTr t;
      double sgn;
      if (face == 0) {          // east r-face (i+1/2, j)
        if (i >= L.nr) continue;
        kL = k; kR = k + 1; g = (i + 0.5) * L.dzc[j]; t = tr_rface(L, tr, V, j, i); sgn = 1.0;
      } else if (face == 1) {   // west r-face (i-1/2, j)
        if (i == 0) continue;
        kL = k - 1; kR = k; g = (i - 0.5) * L.dzc[j]; t = tr_rface(L, tr, V, j, i - 1); sgn = -1.0;
      } else if (face == 2) {   // north z-face (i, j+1/2)
        kL = k; kR = k + P; g = L.volr[i] / L.dz[j]; t = tr_zface(L, tr, V, j, i); sgn = 1.0;
      } else {                  // south z-face (i, j-1/2)
        kL = k - P; kR = k; g = L.volr[i] / L.dz[j - 1]; t = tr_zface(L, tr, V, j - 1, i); sgn = -1.0;
      }
      const double dV = V[kR] - V[kL];
      const double pe = sg_flux(g, t.mu_e, t.D_e, -1.0, ne[kL], ne[kR], dV);
      const double pp = sg_flux(g, t.mu_p, t.D_p, 1.0, np[kL], np[kR], dV);
      const double ps = g * dV;
      Fe += sgn * pe; Fp += sgn * pp; FV += sgn * ps;
      Te += fabs(pe); Tp += fabs(pp); TV += fabs(ps);
    }
    FV += A * kKappa * (np[k] - ne[k]);
    TV += A * kKappa * (fabs(np[k]) + fabs(ne[k]));
    if (write_f) {
      const size_t kf = cidx(P, i, j);
      L.f[NE][kf] = -Fe; L.f[NP][kf] = -Fp; L.f[NV][kf] = -FV;
    }
    if (F0) { F0[k] = Fe; F1[k] = Fp; F2[k] = FV; }
    acc[0] = Fe * Fe; acc[1] = Fp * Fp; acc[2] = FV * FV;
    acc[3] = Te * Te; acc[4] = Tp * Tp; acc[5] = TV * TV;
  }
  reduce_finish<6>(acc, partials, counter, out6, 0);
}

cudaError_t launch_residual(const Level &L, const StateView &sv, const Transport &tr, double dt, bool write_f,
                            double *Fout[3], double *partials, unsigned *counter, double *out6, cudaStream_t st) {
  dim3 b(BX, BY), g((L.nr + 1 + BX - 1) / BX, (L.nz - 1 + BY - 1) / BY);
  k_residual<<<g, b, 0, st>>>(L, sv, tr, dt > 0 ? 1.0 / dt : 0.0, write_f ? 1 : 0, Fout ? Fout[0] : nullptr,
                              Fout ? Fout[1] : nullptr, Fout ? Fout[2] : nullptr, partials, counter, out6);
  count_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Diagonal-block factors (once per Newton iteration and level).  The diagonal block of eq. 14
// at an unknown node is [[a11, 0, a13], [0, a22, a23], [-ak, ak, a33]] with
//   a11 = A/dt + sum(cG over faces where the node is the lower end) + sum(cF where upper),
//   a13 = -sum(cV_e over the four faces), a33 = -sum(g), ak = A e/eps0 (ions likewise),
// and is solved through its Schur complement in V:
//   xV = (rV - q1 re - q2 rp) / s,  s = a33 - q1 a13 - q2 a23,  q1 = -ak/a11,  q2 = ak/a22.
__device__ __forceinline__ void factor_node(const Level &L, const LevelT<float> &M, int mixed, double dt_inv,
                                            double n0, int i, int j) {
  const int P = L.P;
  const size_t k = (size_t)j * P + i;
  const double A = L.volr[i] * L.dzc[j];
  double a11 = A * dt_inv, a22 = A * dt_inv, a13 = 0.0, a23 = 0.0, a33 = 0.0;
  if (i < L.nr) {
    a11 += L.cr[CGE][k]; a22 += L.cr[CGP][k]; a13 -= L.cr[CVE][k]; a23 -= L.cr[CVP][k]; a33 -= L.gR[k];
  }
  if (i > 0) {
    a11 += L.cr[CFE][k - 1]; a22 += L.cr[CFP][k - 1]; a13 -= L.cr[CVE][k - 1]; a23 -= L.cr[CVP][k - 1];
    a33 -= L.gR[k - 1];
  }
  a11 += L.cz[CGE][k]; a22 += L.cz[CGP][k]; a13 -= L.cz[CVE][k]; a23 -= L.cz[CVP][k]; a33 -= L.gZ[k];
  a11 += L.cz[CFE][k - P]; a22 += L.cz[CFP][k - P]; a13 -= L.cz[CVE][k - P]; a23 -= L.cz[CVP][k - P];
  a33 -= L.gZ[k - P];
  const double ak = L.Ak[k];
  const double i11 = 1.0 / a11, i22 = 1.0 / a22;
  const double q1 = -ak * i11, q2 = ak * i22;
  const double is = 1.0 / (a33 - q1 * a13 - q2 * a23);
  const size_t kf = cidx(P, i, j);
  L.fac[FI11][kf] = i11; L.fac[FI22][kf] = i22; L.fac[FQ1][kf] = q1; L.fac[FQ2][kf] = q2; L.fac[FIS][kf] = is;
  L.fac[FA13][kf] = a13; L.fac[FA23][kf] = a23;
  L.dia[DA11][k] = a11; L.dia[DA22][k] = a22; L.dia[DA33][k] = a33;
  if (mixed) {  // density unknowns and rows in units of n0: a13, a23 / n0; q1, q2 * n0
    M.fac[FI11][kf] = (float)i11; M.fac[FI22][kf] = (float)i22;
    M.fac[FQ1][kf] = (float)(q1 * n0); M.fac[FQ2][kf] = (float)(q2 * n0); M.fac[FIS][kf] = (float)is;
    M.fac[FA13][kf] = (float)(a13 / n0); M.fac[FA23][kf] = (float)(a23 / n0);
    M.dia[DA11][k] = (float)a11; M.dia[DA22][k] = (float)a22; M.dia[DA33][k] = (float)a33;
  }
}

__global__ void k_factor(Level L, LevelT<float> M, int mixed, double dt_inv, double n0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
  if (i >= L.ni || j >= L.nz) return;
  factor_node(L, M, mixed, dt_inv, n0, i, j);
}

// Mixed form: FP64 face coefficients of node (i, j) -> FP32 copies in the n0-scaled unknowns
// (density unknowns and density rows divided by n0: cG, cF unchanged, cV / n0).
__device__ __forceinline__ void coef_to32_node(const Level &L, const LevelT<float> &M, double inv_n0, size_t k) {
#pragma unroll
  for (int c = 0; c < NCOEF; ++c) {
    const double sc = (c == CVE || c == CVP) ? inv_n0 : 1.0;
    M.cr[c][k] = (float)(L.cr[c][k] * sc);
    M.cz[c][k] = (float)(L.cz[c][k] * sc);
  }
}

// Levels a .. b in one launch: diagonal factors of the unknown rows and, mixed, the FP32
// coefficient copies of every row.
__global__ void __launch_bounds__(32 * CBY) k_factor_levels(const LevelSet *__restrict__ S, int a, int mixed,
                                                            double dt_inv, double n0) {
  const int l = a + blockIdx.z;
  const Level &L = S->L[l];
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * CBY + threadIdx.y;
  if (i > L.nr || j > L.nz) return;
  if (mixed) coef_to32_node(L, S->M[l], 1.0 / n0, (size_t)j * L.P + i);
  if (j >= 1 && j < L.nz && i < L.ni) factor_node(L, S->M[l], mixed, dt_inv, n0, i, j);
}

cudaError_t launch_factor_levels(const LevelSet *S, const Level &La, int a, int b, bool mixed, double dt, double n0,
                                 cudaStream_t st) {
  if (b < a) return cudaSuccess;
  dim3 bl(32, CBY), g((La.nr + 1 + 31) / 32, (La.nz + 1 + CBY - 1) / CBY, b - a + 1);
  k_factor_levels<<<g, bl, 0, st>>>(S, a, mixed ? 1 : 0, dt > 0 ? 1.0 / dt : 0.0, n0);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_factor(const Level &L, const LevelT<float> *M, double dt, double n0, cudaStream_t st) {
  dim3 b(32, 4), g((L.nr + 1 + 31) / 32, (L.nz - 1 + 3) / 4);
  k_factor<<<g, b, 0, st>>>(L, M ? *M : LevelT<float>(), M ? 1 : 0, dt > 0 ? 1.0 / dt : 0.0, n0);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
struct Triple {
  T e, p, V;
};

__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// One face's share of r = f - (off-diagonal block of eq. 14) x v at a node.  The off-diagonal
// blocks have 5 nonzeros: towards a neighbour across a face where this node is the lower end:
// [-cF, cV] for each species, g for V; where it is the upper end: [-cG, cV], g (cx below is
// cF or cG).  Each product goes into its row with one fused multiply-add: five per face, the
// FP64 pipe being the scarce unit on this GPU.  Electrode-row neighbours carry v = 0.  No
// branches at i = 0, nr: the face arrays hold zeros on the r-faces at i = nr and in the pitch
// padding (never written), so those terms add exact zeros and every load can be issued at once.
template <typename T>
__device__ __forceinline__ void acc_face(T &re, T &rp, T &rV, T cve, T cxe, T cvp, T cxp, T g, T e, T p, T w) {
  re = fmadd(-cve, w, re); re = fmadd(cxe, e, re);
  rp = fmadd(-cvp, w, rp); rp = fmadd(cxp, p, rp);
  rV = fmadd(-g, w, rV);
}

// Solve of the diagonal block through its Schur complement in V (stored factors, see
// factor_node): seven operations.
template <typename T>
__device__ __forceinline__ Triple<T> block_solve(T re, T rp, T rV, T q1, T q2, T is, T a13, T a23, T i11,
                                                 T i22) {
  Triple<T> x;
  x.V = fmadd(-q2, rp, fmadd(-q1, re, rV)) * is;
  x.e = fmadd(-a13, x.V, re) * i11;
  x.p = fmadd(-a23, x.V, rp) * i22;
  return x;
}

// K3: red-black collective Gauss-Seidel half sweep: every node of one colour (red = (i + j)
// even) solves its 3x3 diagonal block (stored factors) against the current neighbours.
// Every operand is loaded before the arithmetic starts (the compiler barrier keeps the loads
// together), so one node costs one round of memory latency; the arithmetic is node_update's,
// term for term: 20 fused multiply-adds for the four faces, 7 for the block solve.
// PDL: the operator data (constant during a linear solve) is requested before waiting for the
// previous kernel, the corrections and right-hand sides after.
// a correction read: through L2 (CG) where another CTA of the same launch wrote it
template <bool CG, typename T> __device__ __forceinline__ T ld_du(const T *p) {
  if (CG) return __ldcg(p);
  return *p;
}

template <typename T, bool PDL = false, bool CG = false>
__device__ __forceinline__ void smooth_node(const LevelT<T> &L, int i, int j) {
  const int P = L.P;
  const size_t k = (size_t)j * P + i;
  const size_t kW = k - 1, kS = k - P;
  const T aE0 = L.cr[CVE][k], aE1 = L.cr[CFE][k], aE2 = L.cr[CVP][k], aE3 = L.cr[CFP][k], gE = L.gR[k];
  const T aW0 = L.cr[CVE][kW], aW1 = L.cr[CGE][kW], aW2 = L.cr[CVP][kW], aW3 = L.cr[CGP][kW], gW = L.gR[kW];
  const T aN0 = L.cz[CVE][k], aN1 = L.cz[CFE][k], aN2 = L.cz[CVP][k], aN3 = L.cz[CFP][k], gN = L.gZ[k];
  const T aS0 = L.cz[CVE][kS], aS1 = L.cz[CGE][kS], aS2 = L.cz[CVP][kS], aS3 = L.cz[CGP][kS], gS = L.gZ[kS];
  const SplitNb d = split_nb(P, i, j);
  const size_t kf = d.self;
  const T q1 = L.fac[FQ1][kf], q2 = L.fac[FQ2][kf], is = L.fac[FIS][kf];
  const T a13 = L.fac[FA13][kf], a23 = L.fac[FA23][kf], i11 = L.fac[FI11][kf], i22 = L.fac[FI22][kf];
  if (PDL) pdl_wait();
  // corrections in the colour-split layout: the four neighbours are of the other colour
  const size_t dE = d.E, dW = d.W, dN = d.N, dS = d.S;
  const T *ve = L.du[NE], *vp = L.du[NP], *vV = L.du[NV];
  const T eE = ld_du<CG>(ve + dE), pE = ld_du<CG>(vp + dE), wE = ld_du<CG>(vV + dE);
  const T eW = ld_du<CG>(ve + dW), pW = ld_du<CG>(vp + dW), wW = ld_du<CG>(vV + dW);
  const T eN = ld_du<CG>(ve + dN), pN = ld_du<CG>(vp + dN), wN = ld_du<CG>(vV + dN);
  const T eS = ld_du<CG>(ve + dS), pS = ld_du<CG>(vp + dS), wS = ld_du<CG>(vV + dS);
  const T f0 = L.f[NE][kf], f1 = L.f[NP][kf], f2 = L.f[NV][kf];
  asm volatile("" ::: "memory");
  T re = f0, rp = f1, rV = f2;
  acc_face(re, rp, rV, aE0, aE1, aE2, aE3, gE, eE, pE, wE);
  acc_face(re, rp, rV, aW0, aW1, aW2, aW3, gW, eW, pW, wW);
  acc_face(re, rp, rV, aN0, aN1, aN2, aN3, gN, eN, pN, wN);
  acc_face(re, rp, rV, aS0, aS1, aS2, aS3, gS, eS, pS, wS);
  const Triple<T> x = block_solve(re, rp, rV, q1, q2, is, a13, a23, i11, i22);
  L.du[NE][kf] = x.e;
  L.du[NP][kf] = x.p;
  L.du[NV][kf] = x.V;
}

// The t-th unknown node of one colour (red: i + j even), row by row: two consecutive rows
// hold ni nodes of each colour together, so threads map onto the colour's nodes with no idle
// lanes inside a row (one row's colour nodes rarely fill whole warps).  False past the end.
__device__ __forceinline__ bool colour_node(int t, int ni, int nz, int color, int &i, int &j) {
  const int p = t / ni, r = t - p * ni;
  const int j0 = 1 + 2 * p;
  const int par0 = (j0 + color) & 1;   // first i of the colour in row j0
  const int n0 = (ni - par0 + 1) >> 1; // colour nodes in row j0
  if (r < n0) { j = j0; i = 2 * r + par0; }
  else { j = j0 + 1; i = 2 * (r - n0) + (par0 ^ 1); }
  return j < nz;
}
// thread slots of colour_node for a level: nz / 2 row pairs of ni
__host__ __device__ __forceinline__ int colour_slots(int ni, int nz) { return (nz / 2) * ni; }

template <typename T>
__global__ void k_smooth(LevelT<T> L, int color) {
  pdl_launch_dependents();
  int i, j;
  if (!colour_node(blockIdx.x * blockDim.x + threadIdx.x, L.ni, L.nz, color, i, j)) return;
  smooth_node<T, true>(L, i, j);
}

// The same half sweep for small levels (FP64, N <= 128): at most 256 threads per block (the
// autotuner's shapes), and the bound lets the compiler keep all of a node's ~44 operands in
// flight at once (96 registers) instead of fetching them in several dependent rounds.  With
// one or two warps per SM that halves the latency of a launch; on the 257^2 level, where
// many warps share each SM, the default allocation is faster.
template <typename T>
__global__ void __launch_bounds__(256, 1) k_smooth_ilp(LevelT<T> L, int color) {
  pdl_launch_dependents();
  int i, j;
  if (!colour_node(blockIdx.x * blockDim.x + threadIdx.x, L.ni, L.nz, color, i, j)) return;
  smooth_node<T, true>(L, i, j);
}

constexpr int SBX = 32, SBY = 2;  // stencil kernels: small blocks so that coarse levels spread over the SMs

// Launch shape (bx, by) is a tuning knob: one thread per node of the colour (colour_node),
// blocks of bx * by threads.
template <typename T>
cudaError_t launch_smooth(const LevelT<T> &L, int color, cudaStream_t st, int bx, int by) {
  const int nb = bx * by;
  dim3 b(nb), g((colour_slots(L.ni, L.nz) + nb - 1) / nb);
  cudaError_t e;
  if (sizeof(T) == 8 && L.nr <= 128 && bx * by <= 256) e = launch_k((L.pdl & PDL_SMOOTH) != 0, k_smooth_ilp<T>, g, b, 0, st, L, color);
  else e = launch_k((L.pdl & PDL_SMOOTH) != 0, k_smooth<T>, g, b, 0, st, L, color);
  count_launch();
  return e;
}
template cudaError_t launch_smooth<double>(const LevelT<double> &, int, cudaStream_t, int, int);
template cudaError_t launch_smooth<float>(const LevelT<float> &, int, cudaStream_t, int, int);


// ------------------------------------------------------------------------------------------
// z-line Gauss-Seidel, zebra order (even columns, then odd): one thread per column of the
// parity solves the column's block-tridiagonal system (rows 1 .. nz-1, 3x3 blocks of eq. 14)
// exactly by block elimination, its r-neighbours (the other parity) held at their current
// values.  Row j:  Lo_j x_{j-1} + D_j x_j + Up_j x_{j+1} = f_j - (E and W couplings),
// D_j = [[a11, 0, a13], [0, a22, a23], [-ak, ak, a33]], Up_j / Lo_j the north / south face
// blocks [[-c_xe, 0, c_ve], [0, -c_xp, c_vp], [0, 0, g]] (c_x = cF towards the north
// neighbour, cG towards the south one).  Forward: M_j = D_j - Lo_j C_{j-1}, C_j = M_j^-1 Up_j,
// y_j = M_j^-1 (rhs_j - Lo_j y_{j-1}) (kept in scr, 12 planes of (nz+1) x cstride);
// backward: x_j = y_j - C_j x_{j+1}, the electrode rows held at zero.  The form for columns the
// shared-memory kernels below do not take: FP64 columns of more than 512 rows, FP32 ones of more
// than 1,024.

// inverse of a general 3x3 matrix (row-major) by its cofactors
template <typename T>
__device__ __forceinline__ void inv3(const T (&m)[9], T (&r)[9]) {
  const T c00 = m[4] * m[8] - m[5] * m[7], c01 = m[5] * m[6] - m[3] * m[8], c02 = m[3] * m[7] - m[4] * m[6];
  const T id = T(1) / (m[0] * c00 + m[1] * c01 + m[2] * c02);
  r[0] = c00 * id; r[1] = (m[2] * m[7] - m[1] * m[8]) * id; r[2] = (m[1] * m[5] - m[2] * m[4]) * id;
  r[3] = c01 * id; r[4] = (m[0] * m[8] - m[2] * m[6]) * id; r[5] = (m[2] * m[3] - m[0] * m[5]) * id;
  r[6] = c02 * id; r[7] = (m[1] * m[6] - m[0] * m[7]) * id; r[8] = (m[0] * m[4] - m[1] * m[3]) * id;
}

template <typename T>
__global__ void k_zline(LevelT<T> L, int color, T *scr, int cstride) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = 2 * t + color;
  if (i >= L.ni) return;
  const int P = L.P, nz = L.nz;
  const size_t plane = (size_t)(nz + 1) * cstride;
  auto S = [&](int q, int j) -> T & { return scr[q * plane + (size_t)j * cstride + t]; };
  T Cp[9] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)}, yp[3] = {T(0), T(0), T(0)};
  for (int j = 1; j < nz; ++j) {
    const size_t k = (size_t)j * P + i, kW = k - 1, kS = k - P;
    const SplitNb d = split_nb(P, i, j);
    T re = L.f[NE][d.self], rp = L.f[NP][d.self], rV = L.f[NV][d.self];
    acc_face(re, rp, rV, L.cr[CVE][k], L.cr[CFE][k], L.cr[CVP][k], L.cr[CFP][k], L.gR[k], L.du[NE][d.E],
             L.du[NP][d.E], L.du[NV][d.E]);
    acc_face(re, rp, rV, L.cr[CVE][kW], L.cr[CGE][kW], L.cr[CVP][kW], L.cr[CGP][kW], L.gR[kW], L.du[NE][d.W],
             L.du[NP][d.W], L.du[NV][d.W]);
    const T ak = L.Ak[k];
    T M[9] = {L.dia[DA11][k], T(0), L.fac[FA13][d.self], T(0), L.dia[DA22][k], L.fac[FA23][d.self], -ak, ak,
              L.dia[DA33][k]};
    // south block (nonzeros l00, l02, l11, l12, l22) times the previous row's C and y
    const T l00 = -L.cz[CGE][kS], l02 = L.cz[CVE][kS], l11 = -L.cz[CGP][kS], l12 = L.cz[CVP][kS], l22 = L.gZ[kS];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      M[c] -= l00 * Cp[c] + l02 * Cp[6 + c];
      M[3 + c] -= l11 * Cp[3 + c] + l12 * Cp[6 + c];
      M[6 + c] -= l22 * Cp[6 + c];
    }
    re -= l00 * yp[0] + l02 * yp[2];
    rp -= l11 * yp[1] + l12 * yp[2];
    rV -= l22 * yp[2];
    T Mi[9];
    inv3(M, Mi);
    // north block (nonzeros u00, u02, u11, u12, u22)
    const T u00 = -L.cz[CFE][k], u02 = L.cz[CVE][k], u11 = -L.cz[CFP][k], u12 = L.cz[CVP][k], u22 = L.gZ[k];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      Cp[3 * r] = Mi[3 * r] * u00;
      Cp[3 * r + 1] = Mi[3 * r + 1] * u11;
      Cp[3 * r + 2] = Mi[3 * r] * u02 + Mi[3 * r + 1] * u12 + Mi[3 * r + 2] * u22;
      yp[r] = Mi[3 * r] * re + Mi[3 * r + 1] * rp + Mi[3 * r + 2] * rV;
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) S(q, j) = Cp[q];
#pragma unroll
    for (int q = 0; q < 3; ++q) S(9 + q, j) = yp[q];
  }
  T xn[3] = {T(0), T(0), T(0)};
  for (int j = nz - 1; j >= 1; --j) {
    T x[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) x[r] = S(9 + r, j) - (S(3 * r, j) * xn[0] + S(3 * r + 1, j) * xn[1] + S(3 * r + 2, j) * xn[2]);
    const size_t kd = cidx(P, i, j);
    L.du[NE][kd] = x[0]; L.du[NP][kd] = x[1]; L.du[NV][kd] = x[2];
    xn[0] = x[0]; xn[1] = x[1]; xn[2] = x[2];
  }
}

// The same column solves by parallel cyclic reduction: one CTA per column, thread t owns row
// t + 1.  Each round (h = 1, 2, 4, ...) every row publishes D^-1 [Lo | Up | r] (21 values) in
// shared memory and folds in its neighbours h rows away:
//   D <- D - Lo (D^-1 Up)_{j-h} - Up (D^-1 Lo)_{j+h},  r <- r - Lo (D^-1 r)_{j-h} - Up (D^-1 r)_{j+h},
//   Lo <- -Lo (D^-1 Lo)_{j-h},  Up <- -Up (D^-1 Up)_{j+h},
// so the couplings move 2h rows away; after log2(nz) rounds the rows are decoupled and
// x_j = D_j^-1 r_j.  Rows past the column ends couple to the electrode rows (x = 0) and are
// dropped.  nz threads (a power of two, up to 1,024).  The FP32 form: its rounds are short and
// it is bound by their latency; in FP64 the rounds' arithmetic bounds it (every row inverts a
// 3x3 block and forms five 3x3 products per round), and block cyclic reduction (k_line_cr, below)
// does about a sixth of that work.
template <typename T>
__device__ __forceinline__ void mm3(const T (&a)[9], const T *b, T (&c)[9]) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) c[3 * r + q] = a[3 * r] * b[q] + a[3 * r + 1] * b[3 + q] + a[3 * r + 2] * b[6 + q];
}

// One unknown of a z-line (column i, row j; rows 1 .. nz-1): the diagonal block, the blocks to the
// rows below (Lo) and above (Up), zero at the column's ends, and the right-hand side with the
// r-neighbours (the other parity's columns) held at their current corrections.
template <typename T>
__device__ __forceinline__ void zline_row(const LevelT<T> &L, int i, int j, T (&D)[9], T (&Lo)[9], T (&Up)[9],
                                          T (&r)[3]) {
  const int P = L.P, nz = L.nz;
  const size_t k = (size_t)j * P + i, kW = k - 1, kS = k - P;
  const SplitNb d = split_nb(P, i, j);
  T re = L.f[NE][d.self], rp = L.f[NP][d.self], rV = L.f[NV][d.self];
  acc_face(re, rp, rV, L.cr[CVE][k], L.cr[CFE][k], L.cr[CVP][k], L.cr[CFP][k], L.gR[k], L.du[NE][d.E],
           L.du[NP][d.E], L.du[NV][d.E]);
  acc_face(re, rp, rV, L.cr[CVE][kW], L.cr[CGE][kW], L.cr[CVP][kW], L.cr[CGP][kW], L.gR[kW], L.du[NE][d.W],
           L.du[NP][d.W], L.du[NV][d.W]);
  r[0] = re; r[1] = rp; r[2] = rV;
  const T ak = L.Ak[k];
#pragma unroll
  for (int q = 0; q < 9; ++q) { D[q] = T(0); Lo[q] = T(0); Up[q] = T(0); }
  D[0] = L.dia[DA11][k]; D[2] = L.fac[FA13][d.self];
  D[4] = L.dia[DA22][k]; D[5] = L.fac[FA23][d.self];
  D[6] = -ak; D[7] = ak; D[8] = L.dia[DA33][k];
  if (j > 1) {
    Lo[0] = -L.cz[CGE][kS]; Lo[2] = L.cz[CVE][kS]; Lo[4] = -L.cz[CGP][kS]; Lo[5] = L.cz[CVP][kS];
    Lo[8] = L.gZ[kS];
  }
  if (j < nz - 1) {
    Up[0] = -L.cz[CFE][k]; Up[2] = L.cz[CVE][k]; Up[4] = -L.cz[CFP][k]; Up[5] = L.cz[CVP][k]; Up[8] = L.gZ[k];
  }
}

// One unknown of an r-line (row j, column i; columns 0 .. ni-1): the blocks to the west (Lo) and
// east (Up) neighbours, [[-c_xe, 0, c_ve], [0, -c_xp, c_vp], [0, 0, g]] of the r-faces (c_x = cG
// towards the west neighbour, cF towards the east one), zero at the row's ends, and the
// right-hand side with the z-neighbours (rows j +- 1, the other parity) held at their current
// corrections.
template <typename T>
__device__ __forceinline__ void rline_row(const LevelT<T> &L, int i, int j, T (&D)[9], T (&Lo)[9], T (&Up)[9],
                                          T (&r)[3]) {
  const int P = L.P, n = L.ni;
  const size_t k = (size_t)j * P + i, kW = k - 1, kS = k - P;
  const SplitNb d = split_nb(P, i, j);
  T re = L.f[NE][d.self], rp = L.f[NP][d.self], rV = L.f[NV][d.self];
  acc_face(re, rp, rV, L.cz[CVE][k], L.cz[CFE][k], L.cz[CVP][k], L.cz[CFP][k], L.gZ[k], L.du[NE][d.N],
           L.du[NP][d.N], L.du[NV][d.N]);
  acc_face(re, rp, rV, L.cz[CVE][kS], L.cz[CGE][kS], L.cz[CVP][kS], L.cz[CGP][kS], L.gZ[kS], L.du[NE][d.S],
           L.du[NP][d.S], L.du[NV][d.S]);
  r[0] = re; r[1] = rp; r[2] = rV;
  const T ak = L.Ak[k];
#pragma unroll
  for (int q = 0; q < 9; ++q) { D[q] = T(0); Lo[q] = T(0); Up[q] = T(0); }
  D[0] = L.dia[DA11][k]; D[2] = L.fac[FA13][d.self];
  D[4] = L.dia[DA22][k]; D[5] = L.fac[FA23][d.self];
  D[6] = -ak; D[7] = ak; D[8] = L.dia[DA33][k];
  if (i > 0) {
    Lo[0] = -L.cr[CGE][kW]; Lo[2] = L.cr[CVE][kW]; Lo[4] = -L.cr[CGP][kW]; Lo[5] = L.cr[CVP][kW];
    Lo[8] = L.gR[kW];
  }
  if (i < n - 1) {
    Up[0] = -L.cr[CFE][k]; Up[2] = L.cr[CVE][k]; Up[4] = -L.cr[CFP][k]; Up[5] = L.cr[CVP][k]; Up[8] = L.gR[k];
  }
}

template <typename T, int MAXT>
__global__ void __launch_bounds__(MAXT) k_zline_pcr(LevelT<T> L, int color) {
  extern __shared__ __align__(16) unsigned char zl_smem[];
  T *X = reinterpret_cast<T *>(zl_smem);  // [21][nz]
  const int nz = L.nz, P = L.P, tid = threadIdx.x;
  const int i = 2 * blockIdx.x + color;
  const int j = tid + 1;
  const bool row = j < nz;
  T D[9], Lo[9], Up[9], r[3];
#pragma unroll
  for (int q = 0; q < 9; ++q) { D[q] = T(0); Lo[q] = T(0); Up[q] = T(0); }
  r[0] = r[1] = r[2] = T(0);
  if (row) zline_row(L, i, j, D, Lo, Up, r);
  for (int h = 1; h < nz; h <<= 1) {
    if (row) {
      T Di[9], t9[9];
      inv3(D, Di);
      mm3(Di, Lo, t9);
#pragma unroll
      for (int q = 0; q < 9; ++q) X[q * nz + j] = t9[q];
      mm3(Di, Up, t9);
#pragma unroll
      for (int q = 0; q < 9; ++q) X[(9 + q) * nz + j] = t9[q];
#pragma unroll
      for (int q = 0; q < 3; ++q) X[(18 + q) * nz + j] = Di[3 * q] * r[0] + Di[3 * q + 1] * r[1] + Di[3 * q + 2] * r[2];
    }
    __syncthreads();
    if (row) {
      const int m = j - h, p = j + h;
      T nLo[9], nUp[9], a9[9], b9[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) { nLo[q] = T(0); nUp[q] = T(0); }
      if (m >= 1) {
#pragma unroll
        for (int q = 0; q < 9; ++q) { a9[q] = X[q * nz + m]; b9[q] = X[(9 + q) * nz + m]; }
        T c9[9];
        mm3(Lo, b9, c9);  // Lo (D^-1 Up)_m
#pragma unroll
        for (int q = 0; q < 9; ++q) D[q] -= c9[q];
        mm3(Lo, a9, c9);  // Lo (D^-1 Lo)_m
#pragma unroll
        for (int q = 0; q < 9; ++q) nLo[q] = -c9[q];
        const T y0 = X[18 * nz + m], y1 = X[19 * nz + m], y2 = X[20 * nz + m];
#pragma unroll
        for (int q = 0; q < 3; ++q) r[q] -= Lo[3 * q] * y0 + Lo[3 * q + 1] * y1 + Lo[3 * q + 2] * y2;
      }
      if (p < nz) {
#pragma unroll
        for (int q = 0; q < 9; ++q) { a9[q] = X[q * nz + p]; b9[q] = X[(9 + q) * nz + p]; }
        T c9[9];
        mm3(Up, a9, c9);  // Up (D^-1 Lo)_p
#pragma unroll
        for (int q = 0; q < 9; ++q) D[q] -= c9[q];
        mm3(Up, b9, c9);  // Up (D^-1 Up)_p
#pragma unroll
        for (int q = 0; q < 9; ++q) nUp[q] = -c9[q];
        const T y0 = X[18 * nz + p], y1 = X[19 * nz + p], y2 = X[20 * nz + p];
#pragma unroll
        for (int q = 0; q < 3; ++q) r[q] -= Up[3 * q] * y0 + Up[3 * q + 1] * y1 + Up[3 * q + 2] * y2;
      }
#pragma unroll
      for (int q = 0; q < 9; ++q) { Lo[q] = nLo[q]; Up[q] = nUp[q]; }
    }
    __syncthreads();
  }
  if (row) {
    T Di[9];
    inv3(D, Di);
    const size_t kd = cidx(P, i, j);
    L.du[NE][kd] = Di[0] * r[0] + Di[1] * r[1] + Di[2] * r[2];
    L.du[NP][kd] = Di[3] * r[0] + Di[4] * r[1] + Di[5] * r[2];
    L.du[NV][kd] = Di[6] * r[0] + Di[7] * r[1] + Di[8] * r[2];
  }
}

// The same line solves by block cyclic reduction (the FP64 form): rows q = 1 .. n of the line
// (z-lines: q = j, n = nz - 1; r-lines: q = i + 1, n = ni).  Level h = 1, 2, 4, ...: the rows
// q = h (2g + 1) are eliminated, each publishing D^-1 [Lo | Up | r] = [a | c | y]; the rows
// q = 2h (g + 1) fold in their neighbours q -+ h exactly as a round of parallel cyclic reduction
// does, so their couplings move 2h rows away; the level whose rows have no survivor left is
// decoupled (x = y).  Back substitution from the top level down: x_q = y_q - a_q x_{q-h} - c_q x_{q+h}.
// Every row is eliminated once, at its own level: over the whole line about a sixth of the
// arithmetic of parallel cyclic reduction, where every row works in every round.  Three lanes per row, lane rr owning row rr of every 3x3 block (its row of
// D^-1 from the cofactors of column rr, det expanded along that column), keep the warps full
// while the levels shrink; a level of at most kLineG9 rows takes nine lanes per row instead, one
// per block entry, three rows to a warp (lanes 0 .. 26), the cofactors and the rows of D^-1
// exchanged by shuffles: the chain of FP64 instructions one warp issues per level, which bounds
// the small levels, is then half as long.  Shared memory: 30 planes of the rows' current blocks
// [D | Lo | Up | r], then 21 of [a | c | y]; the solution goes to the D planes once the forward
// pass is done.  Threads: 3 ceil(n / 2) (at least n: one per row assembles the system), and at
// least a warp per three rows of the largest nine-lane level.
constexpr int kLineG9 = 12;
template <typename T, bool ZL>
__global__ void __launch_bounds__(768, 1) k_line_cr(LevelT<T> L, int color) {
  extern __shared__ __align__(16) unsigned char lc_smem[];
  T *S = reinterpret_cast<T *>(lc_smem);
  const int n = ZL ? L.nz - 1 : L.ni;
  const int line = ZL ? 2 * blockIdx.x + color : 2 * blockIdx.x + 2 - color;
  T *N = S + 30 * n;
  const int tid = threadIdx.x;
  if (tid < n) {
    T D[9], Lo[9], Up[9], r[3];
    if (ZL)
      zline_row(L, line, tid + 1, D, Lo, Up, r);
    else
      rline_row(L, tid, line, D, Lo, Up, r);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      S[q * n + tid] = D[q];
      S[(9 + q) * n + tid] = Lo[q];
      S[(18 + q) * n + tid] = Up[q];
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) S[(27 + q) * n + tid] = r[q];
  }
  __syncthreads();
  const int g = tid / 3, rr = tid - 3 * g;
  const int c1 = rr == 2 ? 0 : rr + 1, c2 = rr == 0 ? 2 : rr - 1;  // (rr + 1) % 3, (rr + 2) % 3
  // nine-lane layout: group g9 (three per warp), entry (r9, c9) of the row's blocks
  const int lane = tid & 31, l9 = lane % 9;
  const int g9 = lane < 27 ? (tid >> 5) * 3 + lane / 9 : 1 << 30;
  const int r9 = l9 / 3, c9 = l9 - 3 * r9;
  const int a1 = r9 == 2 ? 0 : r9 + 1, a2 = r9 == 0 ? 2 : r9 - 1;  // columns other than r9
  const int k1 = c9 == 2 ? 0 : c9 + 1, k2 = c9 == 0 ? 2 : c9 - 1;  // rows other than c9
  const int base9 = lane - c9;                                      // lane of entry (r9, 0)
  int h = 1;
  for (;; h <<= 1) {
    const int E = (n / h + 1) >> 1, Sv = n / (2 * h);
    if (E <= kLineG9) {
      const unsigned m9 = __ballot_sync(0xffffffffu, g9 < E);
      if (g9 < E) {
        const T *Su = S + h * (2 * g9 + 1) - 1;
        T *Nu = N + h * (2 * g9 + 1) - 1;
        // cofactor C[c9][r9]; det expanded along column r9 from the cofactors of lanes (r9, 0 .. 2)
        const T Ck = Su[(3 * k1 + a1) * n] * Su[(3 * k2 + a2) * n] - Su[(3 * k1 + a2) * n] * Su[(3 * k2 + a1) * n];
        const T C0 = __shfl_sync(m9, Ck, base9), C1 = __shfl_sync(m9, Ck, base9 + 1),
                C2 = __shfl_sync(m9, Ck, base9 + 2);
        const T e = Ck * (T(1) / (Su[r9 * n] * C0 + Su[(3 + r9) * n] * C1 + Su[(6 + r9) * n] * C2));
        const T e0 = __shfl_sync(m9, e, base9), e1 = __shfl_sync(m9, e, base9 + 1), e2 = __shfl_sync(m9, e, base9 + 2);
        Nu[(3 * r9 + c9) * n] = e0 * Su[(9 + c9) * n] + e1 * Su[(12 + c9) * n] + e2 * Su[(15 + c9) * n];
        Nu[(9 + 3 * r9 + c9) * n] = e0 * Su[(18 + c9) * n] + e1 * Su[(21 + c9) * n] + e2 * Su[(24 + c9) * n];
        if (c9 == 0) Nu[(18 + r9) * n] = e0 * Su[27 * n] + e1 * Su[28 * n] + e2 * Su[29 * n];
      }
    } else if (g < E) {
      const T *Su = S + h * (2 * g + 1) - 1;
      T *Nu = N + h * (2 * g + 1) - 1;
      const T d0a = Su[c1 * n], d1a = Su[(3 + c1) * n], d2a = Su[(6 + c1) * n];
      const T d0b = Su[c2 * n], d1b = Su[(3 + c2) * n], d2b = Su[(6 + c2) * n];
      const T d0r = Su[rr * n], d1r = Su[(3 + rr) * n], d2r = Su[(6 + rr) * n];
      // cofactors of column rr (rows k = 0, 1, 2)
      const T C0 = d1a * d2b - d1b * d2a, C1 = d2a * d0b - d2b * d0a, C2 = d0a * d1b - d0b * d1a;
      const T id = T(1) / (d0r * C0 + d1r * C1 + d2r * C2);
      const T e0 = C0 * id, e1 = C1 * id, e2 = C2 * id;  // row rr of D^-1
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Nu[(3 * rr + c) * n] = e0 * Su[(9 + c) * n] + e1 * Su[(12 + c) * n] + e2 * Su[(15 + c) * n];
        Nu[(9 + 3 * rr + c) * n] = e0 * Su[(18 + c) * n] + e1 * Su[(21 + c) * n] + e2 * Su[(24 + c) * n];
      }
      Nu[(18 + rr) * n] = e0 * Su[27 * n] + e1 * Su[28 * n] + e2 * Su[29 * n];
    }
    __syncthreads();
    if (Sv == 0) break;
    if (Sv <= kLineG9) {
      const unsigned m9 = __ballot_sync(0xffffffffu, g9 < Sv);
      if (g9 < Sv) {
        const int u = 2 * h * (g9 + 1) - 1;
        T *Su = S + u;
        const T *Nm = N + (u - h);
        const T L0 = Su[(9 + 3 * r9) * n], L1 = Su[(10 + 3 * r9) * n], L2 = Su[(11 + 3 * r9) * n];
        const T U0 = Su[(18 + 3 * r9) * n], U1 = Su[(19 + 3 * r9) * n], U2 = Su[(20 + 3 * r9) * n];
        T Dv = Su[(3 * r9 + c9) * n], r0 = Su[(27 + r9) * n], nU = T(0);
        const T nL = -(L0 * Nm[c9 * n] + L1 * Nm[(3 + c9) * n] + L2 * Nm[(6 + c9) * n]);
        Dv -= L0 * Nm[(9 + c9) * n] + L1 * Nm[(12 + c9) * n] + L2 * Nm[(15 + c9) * n];
        r0 -= L0 * Nm[18 * n] + L1 * Nm[19 * n] + L2 * Nm[20 * n];
        if (u + h < n) {
          const T *Np = N + (u + h);
          Dv -= U0 * Np[c9 * n] + U1 * Np[(3 + c9) * n] + U2 * Np[(6 + c9) * n];
          nU = -(U0 * Np[(9 + c9) * n] + U1 * Np[(12 + c9) * n] + U2 * Np[(15 + c9) * n]);
          r0 -= U0 * Np[18 * n] + U1 * Np[19 * n] + U2 * Np[20 * n];
        }
        __syncwarp(m9);  // the row's blocks are read by all nine lanes before any is overwritten
        Su[(3 * r9 + c9) * n] = Dv;
        Su[(9 + 3 * r9 + c9) * n] = nL;
        Su[(18 + 3 * r9 + c9) * n] = nU;
        if (c9 == 0) Su[(27 + r9) * n] = r0;
      }
    } else if (g < Sv) {
      const int u = 2 * h * (g + 1) - 1;
      T *Su = S + u;
      const T *Nm = N + (u - h);
      T Lr[3], Ur[3], Dr[3], nL[3], nU[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        Lr[k] = Su[(9 + 3 * rr + k) * n];
        Ur[k] = Su[(18 + 3 * rr + k) * n];
        Dr[k] = Su[(3 * rr + k) * n];
      }
      T r0 = Su[(27 + rr) * n];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        nL[c] = -(Lr[0] * Nm[c * n] + Lr[1] * Nm[(3 + c) * n] + Lr[2] * Nm[(6 + c) * n]);
        Dr[c] -= Lr[0] * Nm[(9 + c) * n] + Lr[1] * Nm[(12 + c) * n] + Lr[2] * Nm[(15 + c) * n];
        nU[c] = T(0);
      }
      r0 -= Lr[0] * Nm[18 * n] + Lr[1] * Nm[19 * n] + Lr[2] * Nm[20 * n];
      if (u + h < n) {
        const T *Np = N + (u + h);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          Dr[c] -= Ur[0] * Np[c * n] + Ur[1] * Np[(3 + c) * n] + Ur[2] * Np[(6 + c) * n];
          nU[c] = -(Ur[0] * Np[(9 + c) * n] + Ur[1] * Np[(12 + c) * n] + Ur[2] * Np[(15 + c) * n]);
        }
        r0 -= Ur[0] * Np[18 * n] + Ur[1] * Np[19 * n] + Ur[2] * Np[20 * n];
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Su[(3 * rr + c) * n] = Dr[c];
        Su[(9 + 3 * rr + c) * n] = nL[c];
        Su[(18 + 3 * rr + c) * n] = nU[c];
      }
      Su[(27 + rr) * n] = r0;
    }
    __syncthreads();
  }
  T *X = S;  // planes 0 .. 2: the solution
  T *du = rr == 0 ? L.du[NE] : rr == 1 ? L.du[NP] : L.du[NV];
  for (; h >= 1; h >>= 1) {
    const int E = (n / h + 1) >> 1;
    if (g < E) {
      const int u = h * (2 * g + 1) - 1;
      const T *Nu = N + u;
      T x = Nu[(18 + rr) * n];
      if (u - h >= 0)
        x -= Nu[(3 * rr) * n] * X[u - h] + Nu[(3 * rr + 1) * n] * X[n + u - h] + Nu[(3 * rr + 2) * n] * X[2 * n + u - h];
      if (u + h < n)
        x -= Nu[(9 + 3 * rr) * n] * X[u + h] + Nu[(10 + 3 * rr) * n] * X[n + u + h] +
             Nu[(11 + 3 * rr) * n] * X[2 * n + u + h];
      X[rr * n + u] = x;
      du[ZL ? cidx(L.P, line, u + 1) : cidx(L.P, u, line)] = x;
    }
    __syncthreads();
  }
}

// shared memory and threads of the cyclic-reduction line kernel for a line of n unknowns
template <typename T>
__host__ __forceinline__ size_t line_cr_smem(int n) { return (size_t)51 * n * sizeof(T); }
__host__ __forceinline__ int line_cr_threads(int n) {
  const int half = (n + 1) / 2;
  return std::max((3 * half + 31) / 32 * 32, 32 * ((std::min(half, kLineG9) + 2) / 3));
}

template <typename T, bool ZL>
cudaError_t launch_line_cr(const LevelT<T> &L, int lines, int color, int n, cudaStream_t st) {
  static std::once_flag raised;
  std::call_once(raised, []() {
    cudaFuncSetAttribute(k_line_cr<T, ZL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)line_cr_smem<T>(kRlineMax));
  });
  k_line_cr<T, ZL><<<lines, line_cr_threads(n), line_cr_smem<T>(n), st>>>(L, color);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zline(const LevelT<T> &L, int color, T *scr, cudaStream_t st) {
  const int n = (L.ni - color + 1) / 2;
  if (n <= 0) return cudaSuccess;
  if constexpr (sizeof(T) == 8) {
    // FP64: block cyclic reduction, columns of up to 512 unknowns (208 KB of shared memory)
    if (L.nz - 1 <= kRlineMax) return launch_line_cr<T, true>(L, n, color, L.nz - 1, st);
  } else if (L.nz <= 1024 && (L.nz & (L.nz - 1)) == 0) {
    // FP32: parallel cyclic reduction, one thread per row, 2^k-row columns up to 1,024 (86 KB of
    // shared memory at 1,024; the limit is raised once per instantiation, call_once because the
    // batched host-thread form launches from several threads)
    const size_t smem = (size_t)21 * L.nz * sizeof(T);
    if (L.nz <= 512) {
      k_zline_pcr<T, 512><<<n, L.nz, smem, st>>>(L, color);
    } else {
      static std::once_flag raised1024;
      std::call_once(raised1024, []() {
        cudaFuncSetAttribute(k_zline_pcr<T, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             21 * 1024 * (int)sizeof(T));
      });
      k_zline_pcr<T, 1024><<<n, L.nz, smem, st>>>(L, color);
    }
    count_launch();
    return cudaGetLastError();
  }
  const int cstride = (L.nr + 2) / 2;
  k_zline<T><<<(n + 63) / 64, 64, 0, st>>>(L, color, scr, cstride);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_zline<double>(const LevelT<double> &, int, double *, cudaStream_t);
template cudaError_t launch_zline<float>(const LevelT<float> &, int, float *, cudaStream_t);

// r-line Gauss-Seidel, zebra order (even rows first, then odd): one CTA per row of the parity
// solves the row's block-tridiagonal system along r (unknown columns 0 .. ni-1) exactly, its
// z-neighbours (rows j +- 1, the other parity) held at their current values: in FP32 by the same
// parallel cyclic reduction as the z-lines, a thread per unknown; in FP64 by block cyclic
// reduction (k_line_cr).  Column i:
// Lo_i x_{i-1} + D_i x_i + Up_i x_{i+1} = f_i - (N and S couplings), the W / E face blocks
// [[-c_xe, 0, c_ve], [0, -c_xp, c_vp], [0, 0, g]] of the r-faces (c_x = cG towards the west
// neighbour, cF towards the east one); the wall column of a Dirichlet wall is not an unknown.
template <typename T, int MAXT>
__global__ void __launch_bounds__(MAXT) k_rline_pcr(LevelT<T> L, int color) {
  extern __shared__ __align__(16) unsigned char rl_smem[];
  T *X = reinterpret_cast<T *>(rl_smem);  // [21][ni]
  const int n = L.ni, P = L.P, t = threadIdx.x;
  const int j = 2 * blockIdx.x + 2 - color;  // color 0: rows 2, 4, ...; color 1: rows 1, 3, ...
  const int i = t;
  const bool node = i < n;
  T D[9], Lo[9], Up[9], r[3];
#pragma unroll
  for (int q = 0; q < 9; ++q) { D[q] = T(0); Lo[q] = T(0); Up[q] = T(0); }
  r[0] = r[1] = r[2] = T(0);
  if (node) rline_row(L, i, j, D, Lo, Up, r);
  for (int h = 1; h < n; h <<= 1) {
    if (node) {
      T Di[9], t9[9];
      inv3(D, Di);
      mm3(Di, Lo, t9);
#pragma unroll
      for (int q = 0; q < 9; ++q) X[q * n + i] = t9[q];
      mm3(Di, Up, t9);
#pragma unroll
      for (int q = 0; q < 9; ++q) X[(9 + q) * n + i] = t9[q];
#pragma unroll
      for (int q = 0; q < 3; ++q) X[(18 + q) * n + i] = Di[3 * q] * r[0] + Di[3 * q + 1] * r[1] + Di[3 * q + 2] * r[2];
    }
    __syncthreads();
    if (node) {
      const int m = i - h, p = i + h;
      T nLo[9], nUp[9], a9[9], b9[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) { nLo[q] = T(0); nUp[q] = T(0); }
      if (m >= 0) {
#pragma unroll
        for (int q = 0; q < 9; ++q) { a9[q] = X[q * n + m]; b9[q] = X[(9 + q) * n + m]; }
        T c9[9];
        mm3(Lo, b9, c9);  // Lo (D^-1 Up)_m
#pragma unroll
        for (int q = 0; q < 9; ++q) D[q] -= c9[q];
        mm3(Lo, a9, c9);  // Lo (D^-1 Lo)_m
#pragma unroll
        for (int q = 0; q < 9; ++q) nLo[q] = -c9[q];
        const T y0 = X[18 * n + m], y1 = X[19 * n + m], y2 = X[20 * n + m];
#pragma unroll
        for (int q = 0; q < 3; ++q) r[q] -= Lo[3 * q] * y0 + Lo[3 * q + 1] * y1 + Lo[3 * q + 2] * y2;
      }
      if (p < n) {
#pragma unroll
        for (int q = 0; q < 9; ++q) { a9[q] = X[q * n + p]; b9[q] = X[(9 + q) * n + p]; }
        T c9[9];
        mm3(Up, a9, c9);  // Up (D^-1 Lo)_p
#pragma unroll
        for (int q = 0; q < 9; ++q) D[q] -= c9[q];
        mm3(Up, b9, c9);  // Up (D^-1 Up)_p
#pragma unroll
        for (int q = 0; q < 9; ++q) nUp[q] = -c9[q];
        const T y0 = X[18 * n + p], y1 = X[19 * n + p], y2 = X[20 * n + p];
#pragma unroll
        for (int q = 0; q < 3; ++q) r[q] -= Up[3 * q] * y0 + Up[3 * q + 1] * y1 + Up[3 * q + 2] * y2;
      }
#pragma unroll
      for (int q = 0; q < 9; ++q) { Lo[q] = nLo[q]; Up[q] = nUp[q]; }
    }
    __syncthreads();
  }
  if (node) {
    T Di[9];
    inv3(D, Di);
    const size_t kd = cidx(P, i, j);
    L.du[NE][kd] = Di[0] * r[0] + Di[1] * r[1] + Di[2] * r[2];
    L.du[NP][kd] = Di[3] * r[0] + Di[4] * r[1] + Di[5] * r[2];
    L.du[NV][kd] = Di[6] * r[0] + Di[7] * r[1] + Di[8] * r[2];
  }
}

// rows of one parity: color 0 the even rows 2, 4, ... < nz, color 1 the odd rows 1, 3, ... < nz;
// rows of at most kRlineMax unknowns (mg_create checks)
template <typename T>
cudaError_t launch_rline(const LevelT<T> &L, int color, cudaStream_t st) {
  const int rows = color == 0 ? (L.nz - 2) / 2 : L.nz / 2;
  if (rows <= 0) return cudaSuccess;
  if (L.ni > kRlineMax) return cudaErrorInvalidValue;
  if constexpr (sizeof(T) == 8) {
    return launch_line_cr<T, false>(L, rows, color, L.ni, st);  // FP64: block cyclic reduction
  } else {
    // FP32: parallel cyclic reduction, a thread per unknown (42 KB of shared memory at most)
    k_rline_pcr<T, kRlineMax><<<rows, (L.ni + 31) / 32 * 32, (size_t)21 * L.ni * sizeof(T), st>>>(L, color);
    count_launch();
    return cudaGetLastError();
  }
}
template cudaError_t launch_rline<double>(const LevelT<double> &, int, cudaStream_t);
template cudaError_t launch_rline<float>(const LevelT<float> &, int, cudaStream_t);

// K3 fused: one full red-black sweep per launch.  A block owns a TX x TY tile of nodes.
// Phase 1 updates the red nodes of the tile and of a one-node ring around it (ring nodes are
// also updated by the neighbouring tiles, with identical inputs and arithmetic), keeping them
// in shared memory; phase 2 updates the tile's black nodes from those red values and writes
// both colours.  The black values of the previous sweep are read from `in`, the new ones go
// to `out` (ping-pong buffers), so no block reads what another block writes in the same
// launch and the result equals two half-sweep launches bit for bit.  Coefficients of a face
// are read by its red end in phase 1 and by its black end in phase 2 (an L1/L2 hit).
template <typename T>
__device__ __forceinline__ Triple<T> node_update(const LevelT<T> &L, int i, int j, size_t k, const Triple<T> &vE,
                                                 const Triple<T> &vW, const Triple<T> &vN, const Triple<T> &vS) {
  const int P = L.P;
  const size_t kW = k - 1, kS = k - P;
  const size_t kf = cidx(P, i, j);
  T re = L.f[NE][kf], rp = L.f[NP][kf], rV = L.f[NV][kf];
  acc_face(re, rp, rV, L.cr[CVE][k], L.cr[CFE][k], L.cr[CVP][k], L.cr[CFP][k], L.gR[k], vE.e, vE.p, vE.V);
  acc_face(re, rp, rV, L.cr[CVE][kW], L.cr[CGE][kW], L.cr[CVP][kW], L.cr[CGP][kW], L.gR[kW], vW.e, vW.p, vW.V);
  acc_face(re, rp, rV, L.cz[CVE][k], L.cz[CFE][k], L.cz[CVP][k], L.cz[CFP][k], L.gZ[k], vN.e, vN.p, vN.V);
  acc_face(re, rp, rV, L.cz[CVE][kS], L.cz[CGE][kS], L.cz[CVP][kS], L.cz[CGP][kS], L.gZ[kS], vS.e, vS.p, vS.V);
  return block_solve(re, rp, rV, L.fac[FQ1][kf], L.fac[FQ2][kf], L.fac[FIS][kf], L.fac[FA13][kf],
                     L.fac[FA23][kf], L.fac[FI11][kf], L.fac[FI22][kf]);
}

template <typename T>
__device__ __forceinline__ Triple<T> gload(T *const v[3], size_t k) {
  Triple<T> t;
  t.e = v[NE][k]; t.p = v[NP][k]; t.V = v[NV][k];
  return t;
}

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX * TY) k_sweep(LevelT<T> L, SweepIO<T> io) {
  pdl_launch_dependents();
  pdl_wait();
  constexpr int EX = TX + 2, EY = TY + 2;
  __shared__ T sr[3][EY][EX];
  const int i0 = blockIdx.x * TX - 1, j0 = blockIdx.y * TY;  // extended-tile origin (node coords)
  const int nr = L.nr, nz = L.nz, P = L.P;
  // phase 1: red nodes of the extended tile from the old black values
  for (int q = threadIdx.x; q < EX * EY; q += TX * TY) {
    const int li = q % EX, lj = q / EX;
    const int i = i0 + li, j = j0 + lj;
    T ve = 0, vp = 0, vV = 0;
    if (i >= 0 && i < L.ni && j >= 1 && j < nz && ((i + j) & 1) == 0) {
      const size_t k = (size_t)j * P + i;
      const SplitNb d = split_nb(P, i, j);
      const Triple<T> x = node_update<T>(L, i, j, k, gload<T>(io.in, d.E), gload<T>(io.in, d.W),
                                         gload<T>(io.in, d.N), gload<T>(io.in, d.S));
      ve = x.e; vp = x.p; vV = x.V;
    }
    sr[NE][lj][li] = ve; sr[NP][lj][li] = vp; sr[NV][lj][li] = vV;
  }
  __syncthreads();
  // phase 2: black nodes of the tile from the new red values; both colours written
  {
    const int li = threadIdx.x % TX + 1, lj = threadIdx.x / TX + 1;
    const int i = i0 + li, j = j0 + lj;
    if (i < L.ni && j >= 1 && j < nz) {
      const size_t k = (size_t)j * P + i;
      Triple<T> x;
      if (((i + j) & 1) == 0) {
        x.e = sr[NE][lj][li]; x.p = sr[NP][lj][li]; x.V = sr[NV][lj][li];
      } else {
        auto at = [&](int a, int b) {
          Triple<T> t;
          t.e = sr[NE][b][a]; t.p = sr[NP][b][a]; t.V = sr[NV][b][a];
          return t;
        };
        x = node_update<T>(L, i, j, k, at(li + 1, lj), at(li - 1, lj), at(li, lj + 1), at(li, lj - 1));
      }
      const size_t kd = cidx(P, i, j);
      io.out[NE][kd] = x.e; io.out[NP][kd] = x.p; io.out[NV][kd] = x.V;
    }
  }
}

template <typename T, int TX, int TY>
cudaError_t launch_sweep_t(const LevelT<T> &L, const SweepIO<T> &io, cudaStream_t st) {
  dim3 g((L.nr + 1 + TX - 1) / TX, (L.nz + TY - 1) / TY);  // rows 1..nz-1 live in [0, nz)
  const cudaError_t e = launch_k((L.pdl & PDL_SMOOTH) != 0, k_sweep<T, TX, TY>, g, dim3(TX * TY), 0, st, L, io);
  count_launch();
  return e;
}

template <typename T>
cudaError_t launch_sweep(const LevelT<T> &L, const SweepIO<T> &io, int shape, cudaStream_t st) {
  switch (shape) {
    case 0: return launch_sweep_t<T, 32, 2>(L, io, st);
    case 1: return launch_sweep_t<T, 32, 4>(L, io, st);
    case 2: return launch_sweep_t<T, 32, 8>(L, io, st);
    case 3: return launch_sweep_t<T, 64, 2>(L, io, st);
    case 4: return launch_sweep_t<T, 64, 4>(L, io, st);
    default: return launch_sweep_t<T, 128, 2>(L, io, st);
  }
}
template cudaError_t launch_sweep<double>(const LevelT<double> &, const SweepIO<double> &, int, cudaStream_t);
template cudaError_t launch_sweep<float>(const LevelT<float> &, const SweepIO<float> &, int, cudaStream_t);

// K4: linear residual r = f - J v (or J v when f is null), optional per-field sums of squares
// (accumulated in FP64).
template <typename T>
__device__ __forceinline__ Triple<T> linres_val(const LevelT<T> &L, int i, int j, const T *v0, const T *v1,
                                                const T *v2, const T *f0, const T *f1, const T *f2) {
  const int P = L.P;
  const size_t k = (size_t)j * P + i, kW = k - 1, kS = k - P;
  // f, the factors and v (a correction) in the colour-split layout, the face arrays by row
  const SplitNb d = split_nb(P, i, j);
  const size_t kf = d.self, dE = d.E, dW = d.W, dN = d.N, dS = d.S;
  T re = f0 ? f0[kf] : T(0), rp = f0 ? f1[kf] : T(0), rV = f0 ? f2[kf] : T(0);
  // diagonal block (eq. 14): [[a11, 0, a13], [0, a22, a23], [-ak, ak, a33]]
  re = fmadd(-L.dia[DA11][k], v0[kf], re); re = fmadd(-L.fac[FA13][kf], v2[kf], re);
  rp = fmadd(-L.dia[DA22][k], v1[kf], rp); rp = fmadd(-L.fac[FA23][kf], v2[kf], rp);
  rV = fmadd(-L.Ak[k], v1[kf] - v0[kf], rV); rV = fmadd(-L.dia[DA33][k], v2[kf], rV);
  acc_face(re, rp, rV, L.cr[CVE][k], L.cr[CFE][k], L.cr[CVP][k], L.cr[CFP][k], L.gR[k], v0[dE], v1[dE], v2[dE]);
  acc_face(re, rp, rV, L.cr[CVE][kW], L.cr[CGE][kW], L.cr[CVP][kW], L.cr[CGP][kW], L.gR[kW], v0[dW], v1[dW],
           v2[dW]);
  acc_face(re, rp, rV, L.cz[CVE][k], L.cz[CFE][k], L.cz[CVP][k], L.cz[CFP][k], L.gZ[k], v0[dN], v1[dN], v2[dN]);
  acc_face(re, rp, rV, L.cz[CVE][kS], L.cz[CGE][kS], L.cz[CVP][kS], L.cz[CGP][kS], L.gZ[kS], v0[dS], v1[dS],
           v2[dS]);
  // without f the result is -(J v); negation is exact
  if (!f0) { re = -re; rp = -rp; rV = -rV; }
  return Triple<T>{re, rp, rV};
}

template <typename T>
__device__ __forceinline__ Triple<T> linres_node(const LevelT<T> &L, int i, int j, const T *v0, const T *v1,
                                                 const T *v2, const T *f0, const T *f1, const T *f2, T *o0, T *o1,
                                                 T *o2) {
  const Triple<T> r = linres_val<T>(L, i, j, v0, v1, v2, f0, f1, f2);
  const size_t k = (size_t)j * L.P + i;
  o0[k] = r.e; o1[k] = r.p; o2[k] = r.V;
  return r;
}

template <typename T>
__global__ void k_linres(LevelT<T> L, const T *v0, const T *v1, const T *v2, const T *f0, const T *f1, const T *f2,
                         T *o0, T *o1, T *o2, double *partials, unsigned *counter, double *out3) {
  pdl_launch_dependents();
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
  double acc[3] = {0, 0, 0};
  if (i < L.ni && j < L.nz) {
    const Triple<T> r = linres_node<T>(L, i, j, v0, v1, v2, f0, f1, f2, o0, o1, o2);
    acc[0] = (double)r.e * r.e; acc[1] = (double)r.p * r.p; acc[2] = (double)r.V * r.V;
  }
  if (out3) reduce_finish<3>(acc, partials, counter, out3, 0);
}

template <typename T>
cudaError_t launch_linres(const LevelT<T> &L, T *const v[3], T *const f[3], T *out[3], double *partials,
                          unsigned *counter, double *out3, cudaStream_t st) {
  const int bx = 32, by = SBY;
  dim3 b(bx, by), g((L.nr + 1 + bx - 1) / bx, (L.nz - 1 + by - 1) / by);
  const cudaError_t e = launch_k((L.pdl & PDL_NORM) != 0, k_linres<T>, g, b, 0, st, L, (const T *)v[0], (const T *)v[1],
                                 (const T *)v[2], (const T *)(f ? f[0] : nullptr), (const T *)(f ? f[1] : nullptr),
                                 (const T *)(f ? f[2] : nullptr), out[0], out[1], out[2], partials, counter, out3);
  count_launch();
  return e;
}
template cudaError_t launch_linres<double>(const LevelT<double> &, double *const[3], double *const[3], double *[3],
                                           double *, unsigned *, double *, cudaStream_t);
template cudaError_t launch_linres<float>(const LevelT<float> &, float *const[3], float *const[3], float *[3],
                                          double *, unsigned *, double *, cudaStream_t);

// K5: restriction f_c = P^T r (full weighting in the node coordinates), and du_c = 0.
template <typename T>
__device__ __forceinline__ void restrict_node(const LevelT<T> &F, const LevelT<T> &C, int I, int J) {
  const size_t kc = (size_t)J * C.P + I;
  T s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
  for (int dj = -1; dj <= 1; ++dj) {
    const int j = 2 * J + dj;
    const T wz = dj == 0 ? T(1) : (dj < 0 ? F.wz[j] : T(1) - F.wz[j]);
#pragma unroll
    for (int di = -1; di <= 1; ++di) {
      const int i = 2 * I + di;
      if (i < 0 || i >= F.ni) continue;   // Dirichlet wall nodes carry no residual
      const T w = wz * (di == 0 ? T(1) : T(0.5));
      const size_t kf = (size_t)j * F.P + i;
      s0 += w * F.r[NE][kf]; s1 += w * F.r[NP][kf]; s2 += w * F.r[NV][kf];
    }
  }
  const size_t kcf = cidx(C.P, I, J);
  C.f[NE][kcf] = s0; C.f[NP][kcf] = s1; C.f[NV][kcf] = s2;
  C.du[NE][kcf] = T(0); C.du[NP][kcf] = T(0); C.du[NV][kcf] = T(0);
}


// K4+K5 in one launch: a block computes r = f - J du on the fine nodes under a CX x CY tile of
// coarse nodes (plus the one-node ring the full weighting reaches) into shared memory and
// restricts them; r never goes to global memory.  Same per-node arithmetic and summation order
// as linres_node followed by restrict_node.
// One CX x CY tile of coarse nodes from (I0, J0), threads tid of nthr (all of the CTA reach
// its barrier), sr: 3 x (2 CX + 1)(2 CY + 1) values of shared memory.
template <typename T, int CX, int CY>
__device__ __forceinline__ void linres_restrict_tile(const LevelT<T> &F, const LevelT<T> &C, int I0, int J0, int tid,
                                                     int nthr, T *sr) {
  constexpr int FW = 2 * CX + 1, FH = 2 * CY + 1;
  for (int t = tid; t < FW * FH; t += nthr) {
    const int fi = 2 * I0 - 1 + t % FW, fj = 2 * J0 - 1 + t / FW;
    Triple<T> r{T(0), T(0), T(0)};
    if (fi >= 0 && fi < F.ni && fj < F.nz)
      r = linres_val<T>(F, fi, fj, F.du[NE], F.du[NP], F.du[NV], F.f[NE], F.f[NP], F.f[NV]);
    sr[t] = r.e; sr[FH * FW + t] = r.p; sr[2 * FH * FW + t] = r.V;
  }
  __syncthreads();
  for (int t = tid; t < CX * CY; t += nthr) {
    const int I = I0 + t % CX, J = J0 + t / CX;
    if (I >= C.ni || J >= C.nz) continue;
    T s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj) {
      const int j = 2 * J + dj;
      const T wz = dj == 0 ? T(1) : (dj < 0 ? F.wz[j] : T(1) - F.wz[j]);
#pragma unroll
      for (int di = -1; di <= 1; ++di) {
        const int i = 2 * I + di;
        if (i < 0 || i >= F.ni) continue;
        const T w = wz * (di == 0 ? T(1) : T(0.5));
        const int ls = (j - (2 * J0 - 1)) * FW + (i - (2 * I0 - 1));
        s0 += w * sr[ls]; s1 += w * sr[FH * FW + ls]; s2 += w * sr[2 * FH * FW + ls];
      }
    }
    const size_t kcf = cidx(C.P, I, J);
    C.f[NE][kcf] = s0; C.f[NP][kcf] = s1; C.f[NV][kcf] = s2;
    C.du[NE][kcf] = T(0); C.du[NP][kcf] = T(0); C.du[NV][kcf] = T(0);
  }
}

template <typename T, int CX, int CY>
__global__ void __launch_bounds__(((2 * CX + 1) * (2 * CY + 1) + 31) / 32 * 32) k_linres_restrict(LevelT<T> F,
                                                                                                 LevelT<T> C) {
  __shared__ T sr[3 * (2 * CX + 1) * (2 * CY + 1)];
  pdl_launch_dependents();
  pdl_wait();
  linres_restrict_tile<T, CX, CY>(F, C, blockIdx.x * CX, 1 + blockIdx.y * CY, threadIdx.x, blockDim.x, sr);
}

template <typename T>
cudaError_t launch_linres_restrict(const LevelT<T> &F, const LevelT<T> &C, cudaStream_t st) {
  constexpr int CX = 16, CY = 4;  // 33 x 9 fine nodes, one per thread
  dim3 b(((2 * CX + 1) * (2 * CY + 1) + 31) / 32 * 32), g((C.nr + 1 + CX - 1) / CX, (C.nz - 1 + CY - 1) / CY);
  const cudaError_t e = launch_k((F.pdl & PDL_TRANSFER) != 0, k_linres_restrict<T, CX, CY>, g, b, 0, st, F, C);
  count_launch();
  return e;
}
template cudaError_t launch_linres_restrict<double>(const LevelT<double> &, const LevelT<double> &, cudaStream_t);
template cudaError_t launch_linres_restrict<float>(const LevelT<float> &, const LevelT<float> &, cudaStream_t);

// K6: prolongation and correction du_f += P du_c (bilinear in (r, z)).
template <typename T>
__device__ __forceinline__ void prolong_node(const LevelT<T> &C, const LevelT<T> &F, int i, int j) {
  const size_t kf = cidx(F.P, i, j);  // corrections in the colour-split layout
  int J0, J1;
  T w0, w1;
  if (j & 1) { J0 = (j - 1) >> 1; J1 = J0 + 1; w1 = F.wz[j]; w0 = T(1) - w1; }
  else { J0 = J1 = j >> 1; w0 = T(1); w1 = T(0); }
  int I0, I1;
  T v0, v1;
  if (i & 1) { I0 = (i - 1) >> 1; I1 = I0 + 1; v0 = v1 = T(0.5); }
  else { I0 = I1 = i >> 1; v0 = T(1); v1 = T(0); }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const T *c = C.du[q];
    const T a = v0 * c[cidx(C.P, I0, J0)] + v1 * c[cidx(C.P, I1, J0)];
    const T b = v0 * c[cidx(C.P, I0, J1)] + v1 * c[cidx(C.P, I1, J1)];
    F.du[q][kf] += w0 * a + w1 * b;
  }
}

template <typename T>
__global__ void k_prolong_add(LevelT<T> C, LevelT<T> F) {
  pdl_launch_dependents();
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
  if (i >= F.ni || j >= F.nz) return;
  prolong_node<T>(C, F, i, j);
}

template <typename T>
cudaError_t launch_prolong_add(const LevelT<T> &C, const LevelT<T> &F, cudaStream_t st) {
  dim3 b(SBX, SBY), g((F.nr + 1 + SBX - 1) / SBX, (F.nz - 1 + SBY - 1) / SBY);
  const cudaError_t e = launch_k((F.pdl & PDL_TRANSFER) != 0, k_prolong_add<T>, g, b, 0, st, C, F);
  count_launch();
  return e;
}
template cudaError_t launch_prolong_add<double>(const LevelT<double> &, const LevelT<double> &, cudaStream_t);
template cudaError_t launch_prolong_add<float>(const LevelT<float> &, const LevelT<float> &, cudaStream_t);

// Injection of the state (and optionally the old time level and the sources) to the next grid.
__global__ void k_inject(Level F, StateView fs, Level C, StateView cs, int with_old, int with_src) {
  const int I = blockIdx.x * BX + threadIdx.x;
  const int J = blockIdx.y * BY + threadIdx.y;
  if (I > C.nr || J > C.nz) return;
  const size_t kc = (size_t)J * C.P + I, kf = (size_t)(2 * J) * F.P + 2 * I;
#pragma unroll
  for (int q = 0; q < 3; ++q) cs.u[q][kc] = fs.u[q][kf];
  if (with_old) {
#pragma unroll
    for (int q = 0; q < 3; ++q) cs.uold[q][kc] = fs.uold[q][kf];
  }
  if (with_src) {
    ((double *)cs.S[0])[kc] = fs.S[0][kf];
    ((double *)cs.S[1])[kc] = fs.S[1][kf];
  }
}

cudaError_t launch_inject(const Level &F, const StateView &fs, const Level &C, const StateView &cs, bool with_old,
                          bool with_sources, cudaStream_t st) {
  dim3 b(BX, BY), g((C.nr + 1 + BX - 1) / BX, (C.nz + 1 + BY - 1) / BY);
  k_inject<<<g, b, 0, st>>>(F, fs, C, cs, with_old ? 1 : 0, with_sources ? 1 : 0);
  count_launch();
  return cudaGetLastError();
}

// Continuation: bilinear interpolation of (n_e, n_p, V) from the coarse grid to every fine node.
__global__ void k_prolong_state(Level C, StateView cs, Level F, StateView fs) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i > F.nr || j > F.nz) return;
  const size_t kf = (size_t)j * F.P + i;
  int J0, J1;
  double w0, w1;
  if (j & 1) { J0 = (j - 1) >> 1; J1 = J0 + 1; w1 = F.wz[j]; w0 = 1.0 - w1; }
  else { J0 = J1 = j >> 1; w0 = 1.0; w1 = 0.0; }
  int I0, I1;
  double v0, v1;
  if (i & 1) { I0 = (i - 1) >> 1; I1 = I0 + 1; v0 = v1 = 0.5; }
  else { I0 = I1 = i >> 1; v0 = 1.0; v1 = 0.0; }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const double *c = cs.u[q];
    const double a = v0 * c[(size_t)J0 * C.P + I0] + v1 * c[(size_t)J0 * C.P + I1];
    const double b = v0 * c[(size_t)J1 * C.P + I0] + v1 * c[(size_t)J1 * C.P + I1];
    fs.u[q][kf] = w0 * a + w1 * b;
  }
}

cudaError_t launch_prolong_state(const Level &C, const StateView &cs, const Level &F, const StateView &fs,
                                 cudaStream_t st) {
  dim3 b(BX, BY), g((F.nr + 1 + BX - 1) / BX, (F.nz + 1 + BY - 1) / BY);
  k_prolong_state<<<g, b, 0, st>>>(C, cs, F, fs);
  count_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// K7: coarsest level.  Assemble the dense 3-field Jacobian (unknown q = 3 * node + field,
// node = (j - 1) * (nr + 1) + i), scale columns then rows to unit max-abs entry, and invert the
// scaled matrix by Gauss-Jordan elimination with partial pivoting.  One CTA.
constexpr int CT = 256;
constexpr int kSmemGJ = 48;

// Adds the Jacobian entries of the coarsest level into A (row-major, leading dimension ld,
// zeroed by the caller); thread tid of nthr assembles the rows of nodes tid, tid + nthr, ...
__device__ void assemble_coarse(const Level &L, double dt_inv, double *A, int ld, int tid, int nthr) {
  const int W = L.ni;  // unknown columns (node = (j - 1) * W + i)
  const int nn = W * (L.nz - 1);
  for (int node = tid; node < nn; node += nthr) {
    const int j = node / W + 1, i = node % W;
    const size_t k = (size_t)j * L.P + i;
    const double Av = L.volr[i] * L.dzc[j];
    double a11 = Av * dt_inv, a22 = Av * dt_inv, a13 = 0, a23 = 0, a33 = 0;
    const int re = 3 * node, rp = re + 1, rv = re + 2;
    auto put = [&](int row, int col, double v) { A[(size_t)row * ld + col] += v; };
    // east (towards a Dirichlet wall node only the diagonal terms remain)
    if (i < L.nr) {
      const int nb = 3 * (node + 1);
      const double g = (i + 0.5) * L.dzc[j];
      a11 += L.cr[CGE][k]; a13 -= L.cr[CVE][k]; a22 += L.cr[CGP][k]; a23 -= L.cr[CVP][k]; a33 -= g;
      if (i + 1 < W) {
        put(re, nb, -L.cr[CFE][k]); put(re, nb + 2, L.cr[CVE][k]);
        put(rp, nb + 1, -L.cr[CFP][k]); put(rp, nb + 2, L.cr[CVP][k]);
        put(rv, nb + 2, g);
      }
    }
    if (i > 0) {
      const int nb = 3 * (node - 1);
      const size_t kw = k - 1;
      const double g = (i - 0.5) * L.dzc[j];
      a11 += L.cr[CFE][kw]; a13 -= L.cr[CVE][kw]; a22 += L.cr[CFP][kw]; a23 -= L.cr[CVP][kw]; a33 -= g;
      put(re, nb, -L.cr[CGE][kw]); put(re, nb + 2, L.cr[CVE][kw]);
      put(rp, nb + 1, -L.cr[CGP][kw]); put(rp, nb + 2, L.cr[CVP][kw]);
      put(rv, nb + 2, g);
    }
    {
      const double g = L.volr[i] / L.dz[j];
      a11 += L.cz[CGE][k]; a13 -= L.cz[CVE][k]; a22 += L.cz[CGP][k]; a23 -= L.cz[CVP][k]; a33 -= g;
      if (j + 1 < L.nz) {
        const int nb = 3 * (node + W);
        put(re, nb, -L.cz[CFE][k]); put(re, nb + 2, L.cz[CVE][k]);
        put(rp, nb + 1, -L.cz[CFP][k]); put(rp, nb + 2, L.cz[CVP][k]);
        put(rv, nb + 2, g);
      }
    }
    {
      const size_t ks = k - L.P;
      const double g = L.volr[i] / L.dz[j - 1];
      a11 += L.cz[CFE][ks]; a13 -= L.cz[CVE][ks]; a22 += L.cz[CFP][ks]; a23 -= L.cz[CVP][ks]; a33 -= g;
      if (j - 1 >= 1) {
        const int nb = 3 * (node - W);
        put(re, nb, -L.cz[CGE][ks]); put(re, nb + 2, L.cz[CVE][ks]);
        put(rp, nb + 1, -L.cz[CGP][ks]); put(rp, nb + 2, L.cz[CVP][ks]);
        put(rv, nb + 2, g);
      }
    }
    put(re, re, a11); put(re, rv, a13);
    put(rp, rp, a22); put(rp, rv, a23);
    put(rv, re, -Av * kKappa); put(rv, rp, Av * kKappa); put(rv, rv, a33);
  }
}

// n <= 48 unknowns (the usual 5^2-node coarsest level has n = 45): the augmented matrix
// [A | I] (n x 2n) lives in shared memory from assembly to the inverse.  Per pivot column one
// warp finds the pivot, swaps and scales the pivot row, then four threads per row eliminate
// the remaining columns; entries left of the pivot column are never read again and are not
// updated, so the multiplier A[r][col] stays intact during its step (two barriers per column).
// The body, run by CT threads of one CTA (tid = threadIdx.x < CT; others must not call it) on
// shared arrays sAB (kSmemGJ x 2 kSmemGJ doubles), srs, scs (kSmemGJ each) and *sp_.
__device__ void coarse_factor_smem_body(const Level &L, double dt_inv, double *Minv, double *rs, double *cs,
                                        int *flag, double *sAB, double *srs, double *scs, int *sp_) {
  const int n = 3 * L.ni * (L.nz - 1);
  const int W = 2 * n;
  const int tid = threadIdx.x, lane = tid & 31;
  int &sp = *sp_;
  for (int e = tid; e < n * W; e += CT) sAB[e] = 0.0;
  __syncthreads();
  assemble_coarse(L, dt_inv, sAB, W, tid, CT);
  __syncthreads();
  // equilibration: columns, then rows; identity on the right
  if (tid < n) {
    double m = 0.0;
    for (int r = 0; r < n; ++r) m = fmax(m, fabs(sAB[r * W + tid]));
    scs[tid] = m > 0.0 ? 1.0 / m : 1.0;
  }
  __syncthreads();
  if (tid < n) {
    double m = 0.0;
    for (int c = 0; c < n; ++c) m = fmax(m, fabs(sAB[tid * W + c] * scs[c]));
    srs[tid] = m > 0.0 ? 1.0 / m : 1.0;
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += CT) {
    const int r = e / n, c = e - r * n;
    sAB[r * W + c] *= srs[r] * scs[c];
    sAB[r * W + n + c] = (r == c) ? 1.0 : 0.0;
  }
  if (tid < n) { rs[tid] = srs[tid]; cs[tid] = scs[tid]; }
  __syncthreads();
  const int er = tid >> 2, ec = tid & 3;  // elimination: row er, columns col+1+ec, +4, ...
  for (int col = 0; col < n; ++col) {
    if (tid < 32) {  // pivot search, ties: lowest row index
      double best = -1.0;
      int bi = col;
      for (int r = col + lane; r < n; r += 32) {
        const double v = fabs(sAB[r * W + col]);
        if (v > best) { best = v; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (best > 0.0) {
        if (bi != col)
          for (int c = col + lane; c < W; c += 32) {
            const double t = sAB[bi * W + c];
            sAB[bi * W + c] = sAB[col * W + c];
            sAB[col * W + c] = t;
          }
        __syncwarp();
        const double piv = 1.0 / sAB[col * W + col];
        __syncwarp();
        for (int c = col + 1 + lane; c < W; c += 32) sAB[col * W + c] *= piv;
      }
      if (lane == 0) sp = best > 0.0 ? bi : -1;
    }
    __syncthreads();
    if (sp < 0) {
      if (tid == 0) *flag = 1;
      return;
    }
    if (er < n && er != col) {
      const double fr = sAB[er * W + col];
      if (fr != 0.0)
        for (int c = col + 1 + ec; c < W; c += 4) sAB[er * W + c] -= fr * sAB[col * W + c];
    }
    __syncthreads();
  }
  for (int e = tid; e < n * n; e += CT) {
    const int r = e / n, c = e - r * n;
    Minv[e] = sAB[r * W + n + c];
  }
  if (tid == 0) *flag = 0;
}

__global__ void __launch_bounds__(CT) k_coarse_factor_smem(Level L, double dt_inv, double *Minv, double *rs,
                                                           double *cs, int *flag) {
  __shared__ double sAB[kSmemGJ * 2 * kSmemGJ];
  __shared__ double srs[kSmemGJ], scs[kSmemGJ];
  __shared__ int sp;
  coarse_factor_smem_body(L, dt_inv, Minv, rs, cs, flag, sAB, srs, scs, &sp);
}

// Larger coarsest levels: the same steps in global memory (M is n x n scratch).
__global__ void __launch_bounds__(CT) k_coarse_factor(Level L, double dt_inv, double *M, double *Minv,
                                                      double *rs, double *cs, int *flag) {
  const int nn = L.ni * (L.nz - 1);
  const int n = 3 * nn;
  const int tid = threadIdx.x;
  __shared__ double fac[3 * 9 * 9];
  __shared__ double pv[CT];
  __shared__ int pi[CT];
  for (int e = tid; e < n * n; e += CT) { M[e] = 0.0; Minv[e] = 0.0; }
  __syncthreads();
  assemble_coarse(L, dt_inv, M, n, tid, CT);
  __syncthreads();
  // equilibration: columns, then rows
  for (int c = tid; c < n; c += CT) {
    double m = 0.0;
    for (int r = 0; r < n; ++r) m = fmax(m, fabs(M[(size_t)r * n + c]));
    cs[c] = m > 0.0 ? 1.0 / m : 1.0;
  }
  __syncthreads();
  for (int r = tid; r < n; r += CT) {
    double m = 0.0;
    for (int c = 0; c < n; ++c) m = fmax(m, fabs(M[(size_t)r * n + c] * cs[c]));
    rs[r] = m > 0.0 ? 1.0 / m : 1.0;
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += CT) {
    const int r = e / n, c = e % n;
    M[e] *= rs[r] * cs[c];
    Minv[e] = (r == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  // Gauss-Jordan with partial pivoting (ties: lowest row index)
  for (int col = 0; col < n; ++col) {
    double best = -1.0;
    int bi = col;
    for (int r = col + tid; r < n; r += CT) {
      const double v = fabs(M[(size_t)r * n + col]);
      if (v > best) { best = v; bi = r; }
    }
    pv[tid] = best; pi[tid] = bi;
    __syncthreads();
    for (int o = CT / 2; o > 0; o >>= 1) {
      if (tid < o) {
        const double a = pv[tid], b = pv[tid + o];
        if (b > a || (b == a && pi[tid + o] < pi[tid])) { pv[tid] = b; pi[tid] = pi[tid + o]; }
      }
      __syncthreads();
    }
    const int p = pi[0];
    if (pv[0] <= 0.0) { if (tid == 0) *flag = 1; return; }
    if (p != col) {
      for (int c = tid; c < n; c += CT) {
        double t = M[(size_t)p * n + c]; M[(size_t)p * n + c] = M[(size_t)col * n + c]; M[(size_t)col * n + c] = t;
        t = Minv[(size_t)p * n + c]; Minv[(size_t)p * n + c] = Minv[(size_t)col * n + c]; Minv[(size_t)col * n + c] = t;
      }
    }
    __syncthreads();
    const double piv = 1.0 / M[(size_t)col * n + col];
    __syncthreads();
    for (int c = tid; c < n; c += CT) { M[(size_t)col * n + c] *= piv; Minv[(size_t)col * n + c] *= piv; }
    __syncthreads();
    for (int r = tid; r < n; r += CT) fac[r] = (r == col) ? 0.0 : M[(size_t)r * n + col];
    __syncthreads();
    for (int e = tid; e < n * n; e += CT) {
      const int r = e / n, c = e % n;
      const double fr = fac[r];
      if (fr != 0.0) {
        M[e] -= fr * M[(size_t)col * n + c];
        Minv[e] -= fr * Minv[(size_t)col * n + c];
      }
    }
    __syncthreads();
  }
  if (tid == 0) *flag = 0;
}

cudaError_t launch_coarse_factor(const Level &L, double dt, double *M, double *Minv, double *rs, double *cs,
                                 int *flag, cudaStream_t st) {
  const int n = 3 * L.ni * (L.nz - 1);
  if (n > 3 * 9 * 9) return cudaErrorInvalidValue;
  const double dti = dt > 0 ? 1.0 / dt : 0.0;
  if (n <= kSmemGJ) k_coarse_factor_smem<<<1, CT, 0, st>>>(L, dti, Minv, rs, cs, flag);
  else k_coarse_factor<<<1, CT, 0, st>>>(L, dti, M, Minv, rs, cs, flag);
  count_launch();
  return cudaGetLastError();
}

// du = C Minv R f on the coarsest level (one CTA; one thread per unknown).  For the FP32 inner
// cycle of the mixed form the density entries of f and du are in units of n0 (nscale = n0):
// the FP64 inverse acts on unscaled values.
template <typename T>
__device__ __forceinline__ void coarse_solve_block(const LevelT<T> &L, const double *Minv, const double *rs,
                                                   const double *cs, double nscale, int nthreads) {
  const int nn = L.ni * (L.nz - 1);
  const int n = 3 * nn;
  __shared__ double fs[3 * 9 * 9];
  for (int q = threadIdx.x; q < n; q += nthreads) {
    const int node = q / 3, fld = q % 3;
    const int j = node / L.ni + 1, i = node % L.ni;
    const double sc = fld == NV ? 1.0 : nscale;
    // the field's array chosen by selects, not by a runtime index into the view
    const T *fp = fld == NE ? L.f[NE] : (fld == NP ? L.f[NP] : L.f[NV]);
    fs[q] = rs[q] * sc * (double)fp[cidx(L.P, i, j)];
  }
  __syncthreads();
  for (int q = threadIdx.x; q < n; q += nthreads) {
    double x = 0.0;
    for (int c = 0; c < n; ++c) x += Minv[(size_t)q * n + c] * fs[c];
    const int node = q / 3, fld = q % 3;
    const int j = node / L.ni + 1, i = node % L.ni;
    const double sc = fld == NV ? 1.0 : 1.0 / nscale;
    T *dp = fld == NE ? L.du[NE] : (fld == NP ? L.du[NP] : L.du[NV]);
    dp[cidx(L.P, i, j)] = (T)(cs[q] * x * sc);
  }
}

template <typename T>
__global__ void __launch_bounds__(CT) k_coarse_solve(LevelT<T> L, const double *Minv, const double *rs,
                                                     const double *cs, double nscale) {
  coarse_solve_block<T>(L, Minv, rs, cs, nscale, CT);
}

// ------------------------------------------------------------------------------------------
// K8: the coarse part of a V-cycle (levels S.lv[0] .. S.lv[n-1], the last one solved by the
// dense inverse) in one launch of a thread-block cluster: every phase (a half sweep, the
// residual, the restriction, the coarsest solve, a prolongation) is a loop over the level's
// nodes strided across all threads of the cluster, separated by cluster-wide barriers.  It
// calls the same per-node functions in the same order as the per-level kernels, so the result
// is identical to launching them one by one.
// The phases of K8 over threads tid of nth (a cluster's or one CTA's), `bar` separating them;
// the coarsest solve runs on the first CTA (rank0) with its cta_threads threads.
template <typename T, typename Bar>
__device__ __forceinline__ void coarse_cycle_body(const CoarseSet<T> &S, int tid, int nth, bool rank0, int cta_threads,
                                                  Bar bar) {
  auto sweeps = [&](const LevelT<T> &L, int nu) {
    const int slots = colour_slots(L.ni, L.nz);
    for (int it = 0; it < nu; ++it)
      for (int color = 0; color < 2; ++color) {
        for (int t = tid; t < slots; t += nth) {
          int i, j;
          if (colour_node(t, L.ni, L.nz, color, i, j)) smooth_node<T>(L, i, j);
        }
        bar();
      }
  };
  for (int q = 0; q + 1 < S.n; ++q) {
    const LevelT<T> &L = S.lv[q];
    const LevelT<T> &C = S.lv[q + 1];
    sweeps(L, S.nu1[q]);
    const int W = L.ni;
    for (int t = tid; t < (L.nz - 1) * W; t += nth) {
      const int j = t / W + 1, i = t % W;
      linres_node<T>(L, i, j, L.du[NE], L.du[NP], L.du[NV], L.f[NE], L.f[NP], L.f[NV], L.r[NE], L.r[NP], L.r[NV]);
    }
    bar();
    const int Wc = C.ni;
    for (int t = tid; t < (C.nz - 1) * Wc; t += nth) restrict_node<T>(L, C, t % Wc, t / Wc + 1);
    bar();
  }
  if (rank0) coarse_solve_block<T>(S.lv[S.n - 1], S.Minv, S.rs, S.cs, S.nscale, cta_threads);
  bar();
  for (int q = S.n - 2; q >= 0; --q) {
    const LevelT<T> &F = S.lv[q];
    const int W = F.ni;
    for (int t = tid; t < (F.nz - 1) * W; t += nth) prolong_node<T>(S.lv[q + 1], F, t % W, t / W + 1);
    bar();
    sweeps(F, S.nu2[q]);
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_coarse_cycle(const CoarseSet<T> *__restrict__ sp) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const CoarseSet<T> &S = *sp;
  const int nth = (int)(cl.num_blocks() * blockDim.x);
  const int tid = (int)(cl.block_rank() * blockDim.x + threadIdx.x);
  // barrier.cluster.arrive / wait default to release / acquire at cluster scope, which orders
  // the global-memory writes of one phase before the reads of the next for every CTA of the
  // cluster; a single-CTA set uses the block barrier
  const bool one = cl.num_blocks() == 1;
  coarse_cycle_body<T>(S, tid, nth, cl.block_rank() == 0, (int)blockDim.x, [&]() {
    if (one) __syncthreads();
    else cl.sync();
  });
}

// Single-CTA form of K8 with every array of the coarse levels in shared memory: the
// coefficient, factor and conductance arrays are copied in at the start (constant during a
// linear solve), so are the corrections and the right-hand side of the first level, and its
// correction is copied back at the end (the prolongation to the next finer level reads it).  The phases are those of k_coarse_cycle; what changes is only where the
// arrays live, which turns each phase's dependent global-memory reads into shared-memory ones.
constexpr int kCoarseFields = 2 * NCOEF + NFAC + NDIA + 3 + 9;  // + gR gZ Ak, du f r

template <typename T>
size_t coarse_smem_bytes(const CoarseSet<T> &S) {
  size_t n = 0;
  for (int q = 0; q < S.n; ++q) n += (size_t)(S.lv[q].nz + 1) * S.lv[q].P;
  return n * kCoarseFields * sizeof(T);
}

template <typename T>
__global__ void __launch_bounds__(1024) k_coarse_cycle_smem(const CoarseSet<T> *__restrict__ sp) {
  extern __shared__ __align__(16) unsigned char cc_smem[];
  // per level: offset of its block of kCoarseFields arrays in cc_smem (elements), array length,
  // sizes; the views below derive every array pointer from cc_smem itself, so the compiler
  // addresses them as shared memory (no pointer loads, no generic loads)
  __shared__ int s_off[kMaxCoarseSet], s_len[kMaxCoarseSet], s_nr[kMaxCoarseSet], s_nz[kMaxCoarseSet],
      s_P[kMaxCoarseSet], s_ni[kMaxCoarseSet];
  __shared__ const T *s_wz[kMaxCoarseSet];
  // the coarsest level's dense inverse and scalings when they fit (constant per Newton iteration)
  constexpr int kInvMax = 27;
  __shared__ double s_minv[kInvMax * kInvMax], s_rs[kInvMax], s_cs[kInvMax];
  const CoarseSet<T> &G = *sp;
  const int tid = threadIdx.x, nth = blockDim.x;
  pdl_launch_dependents();
  if (tid == 0) {
    int off = 0;
    for (int q = 0; q < G.n; ++q) {
      const LevelT<T> &g = G.lv[q];
      const int len = (g.nz + 1) * g.P;
      s_off[q] = off; s_len[q] = len; s_nr[q] = g.nr; s_nz[q] = g.nz; s_P[q] = g.P; s_ni[q] = g.ni;
      s_wz[q] = g.wz;
      off += kCoarseFields * len;
    }
  }
  __syncthreads();
  auto view = [&](int q) {
    LevelT<T> v = {};
    v.nr = s_nr[q]; v.nz = s_nz[q]; v.P = s_P[q]; v.ni = s_ni[q]; v.wz = s_wz[q];
    T *b = reinterpret_cast<T *>(cc_smem) + s_off[q];
    const int n = s_len[q];
#pragma unroll
    for (int a = 0; a < NCOEF; ++a) { v.cr[a] = b + a * n; v.cz[a] = b + (NCOEF + a) * n; }
#pragma unroll
    for (int a = 0; a < NFAC; ++a) v.fac[a] = b + (2 * NCOEF + a) * n;
#pragma unroll
    for (int a = 0; a < NDIA; ++a) v.dia[a] = b + (2 * NCOEF + NFAC + a) * n;
    constexpr int g0 = 2 * NCOEF + NFAC + NDIA;
    v.gR = b + g0 * n; v.gZ = b + (g0 + 1) * n; v.Ak = b + (g0 + 2) * n;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      v.du[a] = b + (g0 + 3 + 3 * a) * n; v.f[a] = b + (g0 + 4 + 3 * a) * n; v.r[a] = b + (g0 + 5 + 3 * a) * n;
    }
    return v;
  };
  // copy-in with asynchronous 16-byte copies (every array is a multiple of 16 bytes long and
  // 16-byte aligned at both ends), all issued before one wait: the operator arrays (constant
  // during a linear solve) before waiting for the previous kernel, corrections and right-hand
  // side after
  auto copy = [&](const T *dst, const T *src, int chunks) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    const char *sp = reinterpret_cast<const char *>(src);
    for (int c = tid; c < chunks; c += nth)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d + 16u * c), "l"(sp + 16 * (size_t)c)
                   : "memory");
  };
  auto chunks_of = [&](const LevelT<T> &g) { return (int)((size_t)(g.nz + 1) * g.P * sizeof(T) / 16); };
  for (int q = 0; q < G.n; ++q) {
    const LevelT<T> &g = G.lv[q];
    const LevelT<T> v = view(q);
    const int ch = chunks_of(g);
#pragma unroll
    for (int a = 0; a < NCOEF; ++a) { copy(v.cr[a], g.cr[a], ch); copy(v.cz[a], g.cz[a], ch); }
#pragma unroll
    for (int a = 0; a < NFAC; ++a) copy(v.fac[a], g.fac[a], ch);
#pragma unroll
    for (int a = 0; a < NDIA; ++a) copy(v.dia[a], g.dia[a], ch);
    copy(v.gR, g.gR, ch); copy(v.gZ, g.gZ, ch); copy(v.Ak, g.Ak, ch);
  }
  const LevelT<T> &gc = G.lv[G.n - 1];
  const int nc = 3 * gc.ni * (gc.nz - 1);   // unknowns of the coarsest level
  const bool inv_smem = nc <= kInvMax;
  if (inv_smem) {
    for (int e = tid; e < nc * nc; e += nth) s_minv[e] = G.Minv[e];
    for (int e = tid; e < nc; e += nth) { s_rs[e] = G.rs[e]; s_cs[e] = G.cs[e]; }
  }
  pdl_wait();
  for (int q = 0; q < G.n; ++q) {
    const LevelT<T> &g = G.lv[q];
    const LevelT<T> v = view(q);
    const int ch = chunks_of(g);
    // the first level's correction is the current iterate when the set's first level is the
    // root of the solve; the coarser ones are overwritten by the restriction except for their
    // (zero) electrode rows
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (q == 0) copy(v.f[a], g.f[a], ch);
      copy(v.du[a], g.du[a], ch);
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  // colour nodes packed onto the first warps (colour_node): on 17^2 each colour fills exactly
  // four warps, one per sub-partition, and FP64 issue time goes by warps, not by active lanes
  auto sweeps = [&](const LevelT<T> &L, int nu) {
    const int slots = colour_slots(L.ni, L.nz);
    for (int it = 0; it < nu; ++it)
      for (int color = 0; color < 2; ++color) {
        for (int t = tid; t < slots; t += nth) {
          int i, j;
          if (colour_node(t, L.ni, L.nz, color, i, j)) smooth_node<T>(L, i, j);
        }
        __syncthreads();
      }
  };
  for (int q = 0; q + 1 < G.n; ++q) {
    const LevelT<T> L = view(q);
    const LevelT<T> C = view(q + 1);
    sweeps(L, G.nu1[q]);
    const int W = L.ni;
    for (int t = tid; t < (L.nz - 1) * W; t += nth) {
      const int j = t / W + 1, i = t % W;
      linres_node<T>(L, i, j, L.du[NE], L.du[NP], L.du[NV], L.f[NE], L.f[NP], L.f[NV], L.r[NE], L.r[NP], L.r[NV]);
    }
    __syncthreads();
    const int Wc = C.ni;
    for (int t = tid; t < (C.nz - 1) * Wc; t += nth) restrict_node<T>(L, C, t % Wc, t / Wc + 1);
    __syncthreads();
  }
  {
    const LevelT<T> Lc = view(G.n - 1);
    if (inv_smem) coarse_solve_block<T>(Lc, s_minv, s_rs, s_cs, G.nscale, nth);
    else coarse_solve_block<T>(Lc, G.Minv, G.rs, G.cs, G.nscale, nth);
  }
  __syncthreads();
  for (int q = G.n - 2; q >= 0; --q) {
    const LevelT<T> F = view(q);
    const LevelT<T> C = view(q + 1);
    const int W = F.ni;
    for (int t = tid; t < (F.nz - 1) * W; t += nth) prolong_node<T>(C, F, t % W, t / W + 1);
    __syncthreads();
    sweeps(F, G.nu2[q]);
  }
  {
    const LevelT<T> &g = G.lv[0];
    const LevelT<T> v = view(0);
    const int nodes = (g.nz + 1) * g.P;
#pragma unroll
    for (int a = 0; a < 3; ++a)
      for (int e = tid; e < nodes; e += nth) g.du[a][e] = v.du[a][e];
  }
}

template <typename T>
cudaError_t launch_coarse_cycle(const CoarseSet<T> *dev_set, int cluster, int threads, size_t smem_bytes, bool pdl,
                                cudaStream_t st) {
  if (cluster == 1 && smem_bytes > 0) {
    const cudaError_t e = launch_k(pdl, k_coarse_cycle_smem<T>, dim3(1), dim3(threads), smem_bytes, st, dev_set);
    count_launch();
    return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_coarse_cycle<T>, dev_set);
  count_launch();
  return e;
}
template cudaError_t launch_coarse_cycle<double>(const CoarseSet<double> *, int, int, size_t, bool, cudaStream_t);
template cudaError_t launch_coarse_cycle<float>(const CoarseSet<float> *, int, int, size_t, bool, cudaStream_t);

// Shared memory of the single-CTA coarse cycle for a set (0 when it does not fit); sets the
// kernel's dynamic shared-memory limit.
template <typename T>
size_t prepare_coarse_smem(const CoarseSet<T> &S, size_t limit) {
  const size_t b = coarse_smem_bytes(S);
  if (b > limit) return 0;
  if (cudaFuncSetAttribute(k_coarse_cycle_smem<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b) !=
      cudaSuccess)
    return 0;
  return b;
}
template size_t prepare_coarse_smem<double>(const CoarseSet<double> &, size_t);
template size_t prepare_coarse_smem<float>(const CoarseSet<float> &, size_t);

template <typename T>
cudaError_t launch_coarse_solve(const LevelT<T> &L, const double *Minv, const double *rs, const double *cs,
                                double nscale, cudaStream_t st) {
  k_coarse_solve<T><<<1, CT, 0, st>>>(L, Minv, rs, cs, nscale);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_coarse_solve<double>(const LevelT<double> &, const double *, const double *,
                                                 const double *, double, cudaStream_t);
template cudaError_t launch_coarse_solve<float>(const LevelT<float> &, const double *, const double *,
                                                const double *, double, cudaStream_t);

// Newton update u += du on unknown rows; reduces max |dV| and a non-finite indicator.
__device__ __forceinline__ void update_row(const Level &L, const StateView &sv, int i, int j, double (&acc)[2]) {
  acc[0] = 0.0; acc[1] = 0.0;
  if (i < L.ni && j < L.nz) {
    const size_t k = (size_t)j * L.P + i, kd = cidx(L.P, i, j);
    const double a = L.du[NE][kd], b = L.du[NP][kd], c = L.du[NV][kd];
    sv.u[NE][k] += a; sv.u[NP][k] += b; sv.u[NV][k] += c;
    acc[0] = fabs(c);
    acc[1] = (isfinite(a) && isfinite(b) && isfinite(c)) ? 0.0 : 1.0;
  }
}

__global__ void k_update(Level L, StateView sv, double *partials, unsigned *counter, double *out2) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y + 1;
  double acc[2];
  update_row(L, sv, i, j, acc);
  reduce_finish<2>(acc, partials, counter, out2, 1);
}

cudaError_t launch_update(const Level &L, const StateView &sv, double *partials, unsigned *counter, double *out2,
                          cudaStream_t st) {
  dim3 b(BX, BY), g((L.nr + 1 + BX - 1) / BX, (L.nz - 1 + BY - 1) / BY);
  k_update<<<g, b, 0, st>>>(L, sv, partials, counter, out2);
  count_launch();
  return cudaGetLastError();
}

// Dirichlet electrode rows: n_e = n_p = 0, V = V_cathode (j = 0) and V_anode (j = nz).
// Boundary values: electrode rows (n = 0, V = Vc at z = 0 and Va at z = d) and, with a
// Dirichlet wall (Sec. 3), the wall column (n = 0, V linear in z between Vc and Va).
__global__ void k_dirichlet(Level L, StateView sv, double Vc, double Va) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t <= L.nr) {
    const size_t k0 = t, k1 = (size_t)L.nz * L.P + t;
    sv.u[NE][k0] = 0.0; sv.u[NP][k0] = 0.0; sv.u[NV][k0] = Vc;
    sv.u[NE][k1] = 0.0; sv.u[NP][k1] = 0.0; sv.u[NV][k1] = Va;
  }
  if (L.ni == L.nr && t <= L.nz) {
    const size_t kw = (size_t)t * L.P + L.nr;
    sv.u[NE][kw] = 0.0; sv.u[NP][kw] = 0.0; sv.u[NV][kw] = Vc + (Va - Vc) * L.zf[t];
  }
}

cudaError_t launch_dirichlet(const Level &L, const StateView &sv, double Vc, double Va, cudaStream_t st) {
  const int n = (L.nr > L.nz ? L.nr : L.nz) + 1;
  k_dirichlet<<<(n + 127) / 128, 128, 0, st>>>(L, sv, Vc, Va);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
__global__ void k_zero_du(LevelT<T> L) {
  pdl_launch_dependents();
  pdl_wait();
  const int i = blockIdx.x * BX + threadIdx.x;  // every slot of the row (colour-split layout)
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= L.P || j > L.nz) return;
  const size_t k = (size_t)j * L.P + i;
  L.du[NE][k] = T(0); L.du[NP][k] = T(0); L.du[NV][k] = T(0);
}

template <typename T>
cudaError_t launch_zero_du(const LevelT<T> &L, cudaStream_t st) {
  dim3 b(BX, BY), g((L.P + BX - 1) / BX, (L.nz + 1 + BY - 1) / BY);
  const cudaError_t e = launch_k((L.pdl & PDL_OTHER) != 0, k_zero_du<T>, g, b, 0, st, L);
  count_launch();
  return e;
}
template cudaError_t launch_zero_du<double>(const LevelT<double> &, cudaStream_t);
template cudaError_t launch_zero_du<float>(const LevelT<float> &, cudaStream_t);


// Outer FP64 defect of the mixed solve: x += e (e from the FP32 cycle, densities x n0), then
// r = f - J x in FP64, written as the next FP32 right-hand side (densities / n0), with FP64
// per-field sums of squares.  Two passes: the update must be complete before J x is applied.
__global__ void k_mixed_update(Level L, LevelT<float> M, double n0) {
  pdl_launch_dependents();
  pdl_wait();
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y + 1;
  if (i >= L.ni || j >= L.nz) return;
  const size_t k = cidx(L.P, i, j);
  L.du[NE][k] += n0 * (double)M.du[NE][k];
  L.du[NP][k] += n0 * (double)M.du[NP][k];
  L.du[NV][k] += (double)M.du[NV][k];
}

cudaError_t launch_mixed_update(const Level &L, const LevelT<float> &M, double n0, cudaStream_t st) {
  dim3 b(BX, BY), g((L.nr + 1 + BX - 1) / BX, (L.nz - 1 + BY - 1) / BY);
  const cudaError_t e = launch_k((L.pdl & PDL_OTHER) != 0, k_mixed_update, g, b, 0, st, L, M, n0);
  count_launch();
  return e;
}

// Vectors given in the natural row layout (pitch P) -> the colour-split layout of f and du,
// rows 1 .. nz-1; columns i >= ni (a Dirichlet wall) get zero.
__global__ void k_split_rows(Level L, const double *i0, const double *i1, const double *i2, double *o0,
                             double *o1, double *o2) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y + 1;
  if (i > L.nr || j >= L.nz) return;
  const size_t k = (size_t)j * L.P + i, kf = cidx(L.P, i, j);
  const bool in = i < L.ni;
  o0[kf] = in ? i0[k] : 0.0; o1[kf] = in ? i1[k] : 0.0; o2[kf] = in ? i2[k] : 0.0;
}

cudaError_t launch_split_rows(const Level &L, double *const in[3], double *const out[3], cudaStream_t st) {
  dim3 b(BX, BY), g((L.nr + 1 + BX - 1) / BX, (L.nz - 1 + BY - 1) / BY);
  k_split_rows<<<g, b, 0, st>>>(L, in[0], in[1], in[2], out[0], out[1], out[2]);
  count_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Full Newton Jacobian (mu, D functions of |E|, Sec. 2): the residual's change through the
// transport coefficients when the potential moves by w, which the Picard Jacobian of eq. 14
// (mu, D frozen) leaves out.  Per face and species, flux = g D (n_L G(a) - n_R F(a)),
// a = -s (mu/D)(V_R - V_L), so at fixed n and V_R - V_L
//   d flux = g dD (n_L G(a) - n_R F(a)) + g D (n_L G'(a) - n_R F'(a)) da,
//   da = -s (V_R - V_L) (dmu D - mu dD) / D^2,
// dmu, dD = table segment slope x d|E| (zero where the lookup is clamped), and
// d|E| = (E_n dE_n + E_t dE_t) / |E| with the face field components of w (the same stencils as
// the face |E| of the coefficient kernel).  G = B(-a), F = B(a): n_L G' - n_R F' =
// -(n_L B'(-a) + n_R B'(a)).

// Table values and their |E| slopes (divided by the pressure factor).
__device__ __forceinline__ void lookup_slope1(const Transport &tr, double Eabs, FaceTr &v, FaceTr &d) {
  const double *T = tr.table;
  const int n = tr.rows;
  const double E0 = __ldg(T), E1 = __ldg(T + 5 * (n - 1));
  const bool inside = Eabs >= E0 && Eabs <= E1;
  const double x = fmin(fmax(Eabs, E0), E1);
  int lo = 0, hi = n - 1;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(T + 5 * mid) <= x) lo = mid; else hi = mid;
  }
  const double *a = T + 5 * lo, *b = a + 5;
  const double ih = __ldg(tr.inv_dE + lo);
  const double t = (x - __ldg(a)) * ih;
  double sl[4], val[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double ya = __ldg(a + 1 + c), yb = __ldg(b + 1 + c);
    val[c] = (ya + t * (yb - ya)) * tr.inv_pf;
    sl[c] = inside ? (yb - ya) * ih * tr.inv_pf : 0.0;
  }
  v = FaceTr{val[0], val[1], val[2], val[3]};
  d = FaceTr{sl[0], sl[1], sl[2], sl[3]};
}

// d flux of both species through one face; En, Et: the face field components of the state,
// dEn, dEt: those of w; dV = V_R - V_L.
__device__ __forceinline__ Triple<double> face_dflux(const Transport &tr, double g, double En, double Et, double dEn,
                                                     double dEt, double dV, double neL, double neR, double npL,
                                                     double npR) {
  const double Em = sqrt(En * En + Et * Et);
  const double dEm = Em > 0.0 ? (En * dEn + Et * dEt) / Em : 0.0;
  FaceTr t, sl;
  lookup_slope1(tr, Em, t, sl);
  Triple<double> out{0.0, 0.0, 0.0};
  {  // electrons, s = -1: a = (mu/D) dV
    const double a = (t.mu_e / t.D_e) * dV;
    const Bern b = bernoulli1(a);
    const double dmu = sl.mu_e * dEm, dD = sl.D_e * dEm;
    const double da = dV * (dmu * t.D_e - t.mu_e * dD) / (t.D_e * t.D_e);
    out.e = g * dD * (neL * b.Bm - neR * b.Bp) - g * t.D_e * (neL * b.dBm + neR * b.dBp) * da;
  }
  {  // ions, s = +1: a = -(mu/D) dV
    const double a = -(t.mu_p / t.D_p) * dV;
    const Bern b = bernoulli1(a);
    const double dmu = sl.mu_p * dEm, dD = sl.D_p * dEm;
    const double da = -dV * (dmu * t.D_p - t.mu_p * dD) / (t.D_p * t.D_p);
    out.p = g * dD * (npL * b.Bm - npR * b.Bp) - g * t.D_p * (npL * b.dBm + npR * b.dBp) * da;
  }
  return out;
}

// The transport part of (J w) in the two continuity rows of unknown node (i, j); w in the
// colour-split layout of the corrections, the state in row order.
__device__ __forceinline__ Triple<double> transport_row(const Level &L, const StateView &sv, const Transport &tr,
                                                        const double *w, int i, int j) {
  const int P = L.P;
  const size_t k = (size_t)j * P + i;
  const double *ne = sv.u[NE], *np = sv.u[NP], *V = sv.u[NV];
  auto W = [&](int ii, int jj) { return w[cidx(P, ii, jj)]; };
  Triple<double> r{0.0, 0.0, 0.0};
  // r-face between columns c and c + 1 of row j (j interior)
  auto rface = [&](int c) {
    const size_t kL = (size_t)j * P + c, kR = kL + 1;
    const double En = (V[kL] - V[kR]) * L.idr;
    const double lo = (V[kL - P] - V[kL]) + (V[kR - P] - V[kR]);
    const double up = (V[kL] - V[kL + P]) + (V[kR] - V[kR + P]);
    const double Et = 0.25 * (lo * L.idz[j - 1] + up * L.idz[j]);
    const double dEn = (W(c, j) - W(c + 1, j)) * L.idr;
    const double dlo = (W(c, j - 1) - W(c, j)) + (W(c + 1, j - 1) - W(c + 1, j));
    const double dup = (W(c, j) - W(c, j + 1)) + (W(c + 1, j) - W(c + 1, j + 1));
    const double dEt = 0.25 * (dlo * L.idz[j - 1] + dup * L.idz[j]);
    return face_dflux(tr, L.gR[kL], En, Et, dEn, dEt, V[kR] - V[kL], ne[kL], ne[kR], np[kL], np[kR]);
  };
  // z-face between rows q and q + 1 of column i
  auto zface = [&](int q) {
    const size_t kL = (size_t)q * P + i, kR = kL + P;
    const double En = (V[kL] - V[kR]) * L.idz[q];
    const double dEn = (W(i, q) - W(i, q + 1)) * L.idz[q];
    double Et = 0.0, dEt = 0.0;
    if (i > 0 && i < L.nr) {
      Et = 0.25 * L.idr * ((V[kL - 1] - V[kL + 1]) + (V[kR - 1] - V[kR + 1]));
      dEt = 0.25 * L.idr * ((W(i - 1, q) - W(i + 1, q)) + (W(i - 1, q + 1) - W(i + 1, q + 1)));
    }
    return face_dflux(tr, L.gZ[kL], En, Et, dEn, dEt, V[kR] - V[kL], ne[kL], ne[kR], np[kL], np[kR]);
  };
  if (i < L.nr) { const Triple<double> f = rface(i); r.e += f.e; r.p += f.p; }
  if (i > 0) { const Triple<double> f = rface(i - 1); r.e -= f.e; r.p -= f.p; }
  { const Triple<double> f = zface(j); r.e += f.e; r.p += f.p; }
  { const Triple<double> f = zface(j - 1); r.e -= f.e; r.p -= f.p; }
  (void)k;
  return r;
}

// Defect of the full-Jacobian Newton step: f = fs - J_full d (J_full = the Picard operator of
// level L plus the transport part), written as the right-hand side of the next correction
// (colour-split), with its per-field sums of squares.
__global__ void __launch_bounds__(32 * CBY) k_full_defect(Level L, StateView sv, Transport tr, const double *fs0,
                                                          const double *fs1, const double *fs2, const double *d0,
                                                          const double *d1, const double *d2, double *partials,
                                                          unsigned *counter, double *out3) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * CBY + threadIdx.y + 1;
  double acc[3] = {0, 0, 0};
  if (i < L.ni && j < L.nz) {
    Triple<double> r = linres_val<double>(L, i, j, d0, d1, d2, fs0, fs1, fs2);
    if (tr.table) {
      const Triple<double> t = transport_row(L, sv, tr, d2, i, j);
      r.e -= t.e;
      r.p -= t.p;
    }
    const size_t kf = cidx(L.P, i, j);
    L.f[NE][kf] = r.e; L.f[NP][kf] = r.p; L.f[NV][kf] = r.V;
    acc[0] = r.e * r.e; acc[1] = r.p * r.p; acc[2] = r.V * r.V;
  }
  reduce_finish<3>(acc, partials, counter, out3, 0);
}

cudaError_t launch_full_defect(const Level &L, const StateView &sv, const Transport &tr, double *const fs[3],
                               double *const d[3], double *partials, unsigned *counter, double *out3, cudaStream_t st) {
  dim3 b(32, CBY), g((L.nr + 1 + 31) / 32, (L.nz - 1 + CBY - 1) / CBY);
  k_full_defect<<<g, b, 0, st>>>(L, sv, tr, fs[0], fs[1], fs[2], d[0], d[1], d[2], partials, counter, out3);
  count_launch();
  return cudaGetLastError();
}

// out (row layout) += the transport part of J w on the unknown nodes (w colour-split)
__global__ void __launch_bounds__(32 * CBY) k_add_transport(Level L, StateView sv, Transport tr, const double *w,
                                                            double *o0, double *o1) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * CBY + threadIdx.y + 1;
  if (i >= L.ni || j >= L.nz || !tr.table) return;
  const Triple<double> t = transport_row(L, sv, tr, w, i, j);
  const size_t k = (size_t)j * L.P + i;
  o0[k] += t.e;
  o1[k] += t.p;
}

cudaError_t launch_add_transport(const Level &L, const StateView &sv, const Transport &tr, const double *w,
                                 double *out[3], cudaStream_t st) {
  dim3 b(32, CBY), g((L.nr + 1 + 31) / 32, (L.nz - 1 + CBY - 1) / CBY);
  k_add_transport<<<g, b, 0, st>>>(L, sv, tr, w, out[0], out[1]);
  count_launch();
  return cudaGetLastError();
}

// acc += x over n elements of three arrays
__global__ void k_add3(double *a0, double *a1, double *a2, const double *x0, const double *x1, const double *x2,
                       size_t n) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  a0[e] += x0[e]; a1[e] += x1[e]; a2[e] += x2[e];
}

cudaError_t launch_add3(double *const acc[3], double *const x[3], size_t n, cudaStream_t st) {
  k_add3<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(acc[0], acc[1], acc[2], x[0], x[1], x[2], n);
  count_launch();
  return cudaGetLastError();
}

// The colour-split layout -> natural rows, every row 0 .. nz.
__global__ void k_join_rows(Level L, const double *i0, const double *i1, const double *i2, double *o0, double *o1,
                            double *o2) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i > L.nr || j > L.nz) return;
  const size_t k = (size_t)j * L.P + i, kf = cidx(L.P, i, j);
  o0[k] = i0[kf]; o1[k] = i1[kf]; o2[k] = i2[kf];
}

cudaError_t launch_join_rows(const Level &L, double *const in[3], double *const out[3], cudaStream_t st) {
  dim3 b(BX, BY), g((L.nr + 1 + BX - 1) / BX, (L.nz + 1 + BY - 1) / BY);
  k_join_rows<<<g, b, 0, st>>>(L, in[0], in[1], in[2], out[0], out[1], out[2]);
  count_launch();
  return cudaGetLastError();
}

__device__ __forceinline__ void outer_row(const Level &L, const LevelT<float> &M, double inv_n0, int i, int j,
                                          double (&acc)[3]) {
  acc[0] = 0.0; acc[1] = 0.0; acc[2] = 0.0;
  if (i < L.ni && j < L.nz) {
    const Triple<double> r = linres_val<double>(L, i, j, L.du[NE], L.du[NP], L.du[NV], L.f[NE], L.f[NP], L.f[NV]);
    const double re = r.e, rp = r.p, rV = r.V;
    const size_t kf = cidx(L.P, i, j);
    M.f[NE][kf] = (float)(re * inv_n0);
    M.f[NP][kf] = (float)(rp * inv_n0);
    M.f[NV][kf] = (float)rV;
    acc[0] = re * re; acc[1] = rp * rp; acc[2] = rV * rV;
  }
}

__global__ void k_outer_residual(Level L, LevelT<float> M, double inv_n0, double *partials, unsigned *counter,
                                 double *out3) {
  pdl_launch_dependents();
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
  double acc[3];
  outer_row(L, M, inv_n0, i, j, acc);
  reduce_finish<3>(acc, partials, counter, out3, 0);
}

cudaError_t launch_outer_residual(const Level &L, const LevelT<float> &M, double n0, double *partials,
                                  unsigned *counter, double *out3, cudaStream_t st) {
  dim3 b(BX, BY), g((L.nr + 1 + BX - 1) / BX, (L.nz - 1 + BY - 1) / BY);
  const cudaError_t e = launch_k((L.pdl & PDL_NORM) != 0, k_outer_residual, g, b, 0, st, L, M, 1.0 / n0, partials, counter, out3);
  count_launch();
  return e;
}

// ------------------------------------------------------------------------------------------
// Cycle control on the device (row a7): the V-cycle loop of a linear solve runs inside a CUDA
// graph as a conditional WHILE node; these one-thread kernels evaluate the stopping test
//   max_f ||r_f|| / w_f  <=  eta * (the same at du = 0)
// from the per-field sums of squares norm3, record the history and set the loop condition.
__device__ __forceinline__ double weighted_norm(const SolveCtl *c, const double *norm3) {
  double m = 0.0;
  for (int q = 0; q < 3; ++q) {
    const double v = sqrt(norm3[q]) / c->w[q];
    if (!(v == v)) return NAN;
    m = fmax(m, v);
  }
  return m;
}

__global__ void k_solve_init(SolveCtl *c, const double *norm3, cudaGraphConditionalHandle h) {
  const double r0 = weighted_norm(c, norm3);
  c->r0 = r0;
  c->ncyc = 0;
  c->rel = r0 > 0.0 ? 1.0 : 0.0;
  c->hist[0] = c->rel;
  const bool go = r0 > 0.0 && isfinite(r0) && c->rel > c->eta && c->max_cycles > 0;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

__global__ void k_solve_check(SolveCtl *c, const double *norm3, cudaGraphConditionalHandle h) {
  const double rel = weighted_norm(c, norm3) / c->r0;
  const int n = c->ncyc + 1;
  c->ncyc = n;
  c->rel = rel;
  if (n < kMaxHist) c->hist[n] = rel;
  const bool go = isfinite(rel) && rel > c->eta && n < c->max_cycles;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

cudaError_t launch_solve_init(SolveCtl *ctl, const double *norm3, cudaGraphConditionalHandle h, cudaStream_t st) {
  k_solve_init<<<1, 1, 0, st>>>(ctl, norm3, h);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_solve_check(SolveCtl *ctl, const double *norm3, cudaGraphConditionalHandle h, cudaStream_t st) {
  k_solve_check<<<1, 1, 0, st>>>(ctl, norm3, h);
  count_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// FP64 FMA throughput probe: 8 independent FMA chains per thread, enough warps to fill every SM.
__global__ void k_fp64_probe(double *out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = threadIdx.x * 1e-3 + q;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = fma(x[q], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += x[q];
  if (s == 12345.678) out[0] = s;  // keeps the chains live
}

double probe_fp64_gflops(cudaStream_t st) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1.0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1.0;
  double *out = nullptr;
  if (cudaMalloc(&out, sizeof(double)) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sms * 8, threads = 256, iters = 4096;
  k_fp64_probe<<<blocks, threads, 0, st>>>(out, 64, 0.999999, 1e-7);  // warm-up
  cudaEventRecord(e0, st);
  k_fp64_probe<<<blocks, threads, 0, st>>>(out, iters, 0.999999, 1e-7);
  cudaEventRecord(e1, st);
  count_launch(2);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || ms <= 0.f) return -1.0;
  const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
  return flops / (ms * 1e-3) / 1e9;
}

// ------------------------------------------------------------------------------------------
// Batched form (row a11): one persistent launch runs the steady solves of many discharges.
// Each discharge's solve is a state machine (batch_control below: the continuation, the
// Delta-t march with its accept / reject rules, the Newton loop of each step, as the host
// driver runs them for one discharge) whose GPU work is a sequence of phases taken from the
// discharge's program (mg_api.cu builds it from the launches of the single-discharge path).
// The CTAs claim work items (tiles) of any discharge's current phase; the CTA that finishes a
// phase's last tile folds the phase's reductions, lets the state machine choose the next phase
// and publishes it.  No CTA waits for another: a CTA without work looks again (with a growing
// pause), so progress needs no co-residency; if no phase finishes anywhere for kBatchIdleNs a
// CTA marks the launch as failed and every CTA leaves.
//
// Every tile runs the per-node functions of the corresponding single-discharge kernel over
// the same nodes; reductions replicate reduce_finish's per-block partials (virtual blocks of the
// original block shape) and its fold, and the state machine evaluates the host driver's
// expressions operation by operation, so the solves equal the single-discharge ones bit for bit.
//
// Claims: claim = (sequence << 32) | count.  A claimer adds 1; the value returned names the
// phase (ring[sequence & 3] must carry the same sequence) and the tile (count < ntiles).  The
// finisher writes ring[(sequence + 1) & 3], resets done, fences, then swaps in the next
// sequence with count 0; a claim that lands after the swap is a valid claim of the new phase.
// Visibility: tile writes -> CTA barrier -> release-acquire add on `done` (the finisher acquires
// every tile's writes); the publisher's swap of `claim` releases, and a claim (acquire-release
// add) acquires, before any data of earlier phases is read.
constexpr unsigned long long kBatchIdleNs = 5000000000ull;
constexpr int kBW = kBatchThreads / 32;   // warps per CTA

// ring entry: (sequence << 32) | (program counter << 20) | work items of the phase
__device__ __forceinline__ unsigned long long ring_entry(unsigned seq, int pc, int ntiles) {
  return ((unsigned long long)seq << 32) | ((unsigned long long)(unsigned)pc << 20) | (unsigned)ntiles;
}
__device__ __forceinline__ int ring_pc(unsigned long long e) { return (int)((e >> 20) & 0xfffu); }
__device__ __forceinline__ unsigned ring_ntiles(unsigned long long e) { return (unsigned)(e & 0xfffffu); }
__device__ __forceinline__ unsigned long long ld_vol64(const unsigned long long *p) {
  return *reinterpret_cast<const volatile unsigned long long *>(p);
}
// Acquire-release atomics at GPU scope: a claim acquires the publisher's writes (ring entry,
// state machine, data of earlier phases), a finished tile releases its CTA's writes (the CTA
// barrier before it orders them), and the publisher's swap releases the next phase.
__device__ __forceinline__ unsigned long long atom_add_acqrel64(unsigned long long *p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned atom_add_acqrel32(unsigned *p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void atom_exch_release64(unsigned long long *p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.release.gpu.global.exch.b64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  (void)old;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// reduce_finish's block partial for a virtual block of nv threads (nv / 32 consecutive warps of
// the CTA starting at a multiple of nv): warp sums (or maxima), then the block's thread 0 adds
// its warps in order and writes dst[0..K) when `valid`.  Every thread of the CTA calls it.
template <int K>
__device__ __forceinline__ void vblock_partial(const double (&v)[K], int nv, bool valid, double *dst, double *sh,
                                               int op) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    double x = v[q];
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_down_sync(0xffffffffu, x, o);
      x = op ? fmax(x, y) : x + y;
    }
    if (lane == 0) sh[q * kBW + wid] = x;
  }
  __syncthreads();
  if ((tid % nv) == 0 && valid) {
    const int nw = nv >> 5;
#pragma unroll
    for (int q = 0; q < K; ++q) {
      double x = sh[q * kBW + wid];
      for (int w = 1; w < nw; ++w) x = op ? fmax(x, sh[q * kBW + wid + w]) : x + sh[q * kBW + wid + w];
      dst[q] = x;
    }
  }
  __syncthreads();
}

// reduce_finish's last-block fold of nblocks partials by nthr threads (the original block size;
// threads tid >= nthr only pass the barriers), result in out[0..K).
template <int K>
__device__ __forceinline__ void fold_partials(const double *partials, int nblocks, int nthr, double *out,
                                              double *sh, int op) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const bool act = tid < nthr;
  double xs[K];
  bool first = true;
#pragma unroll
  for (int q = 0; q < K; ++q) xs[q] = 0.0;
  if (act) {
    int b = tid;
    for (; b + 3 * nthr < nblocks; b += 4 * nthr) {
      double y[4][K];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < K; ++q) y[u][q] = __ldcg(partials + (size_t)(b + u * nthr) * K + q);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < K; ++q)
          xs[q] = (first && u == 0) ? y[u][q] : (op ? fmax(xs[q], y[u][q]) : xs[q] + y[u][q]);
      first = false;
    }
    for (; b < nblocks; b += nthr) {
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const double y = __ldcg(partials + (size_t)b * K + q);
        xs[q] = first ? y : (op ? fmax(xs[q], y) : xs[q] + y);
      }
      first = false;
    }
  }
#pragma unroll
  for (int q = 0; q < K; ++q) {
    double x = first ? (op ? -1.0 : 0.0) : xs[q];
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_down_sync(0xffffffffu, x, o);
      x = op ? fmax(x, y) : x + y;
    }
    if (lane == 0 && act) sh[q * kBW + wid] = x;
  }
  __syncthreads();
  if (tid == 0) {
    const int nw = nthr >> 5;
#pragma unroll
    for (int q = 0; q < K; ++q) {
      double x = sh[q * kBW];
      for (int w = 1; w < nw; ++w) x = op ? fmax(x, sh[q * kBW + w]) : x + sh[q * kBW + w];
      out[q] = x;
    }
  }
  __syncthreads();
}

// Shared memory of the persistent launch: reduction scratch, then the largest phase buffer (the
// coarsest level's augmented matrix; the restriction tile fits in it too).
constexpr int kBatchRestrCX = 16, kBatchRestrCY = 3;  // 33 x 7 fine nodes per coarse tile: <= 256 threads
constexpr size_t kBatchShRed = 16 * kBW * sizeof(double);
constexpr size_t kBatchShGJ = (size_t)kSmemGJ * 2 * kSmemGJ * sizeof(double) + 2 * kSmemGJ * sizeof(double) + 16;
constexpr size_t kBatchShRestr = 3 * (2 * kBatchRestrCX + 1) * (2 * kBatchRestrCY + 1) * sizeof(double);
constexpr size_t kBatchSmem = kBatchShRed + (kBatchShGJ > kBatchShRestr ? kBatchShGJ : kBatchShRestr);

// 32 x 8 thread block b of a (gx, gy, levels) grid: level offset, node (i, j) of this thread
__device__ __forceinline__ void vb328(int b, int gx, int gy, int &lz, int &i, int &j) {
  const int per = gx * gy;
  lz = b / per;
  const int r = b - lz * per;
  i = (r % gx) * 32 + (threadIdx.x & 31);
  j = (r / gx) * 8 + (threadIdx.x >> 5);
}

template <typename T>
__device__ __forceinline__ const LevelT<T> &lview(const LevelSet *S, int l);
template <>
__device__ __forceinline__ const LevelT<double> &lview<double>(const LevelSet *S, int l) { return S->L[l]; }
template <>
__device__ __forceinline__ const LevelT<float> &lview<float>(const LevelSet *S, int l) { return S->M[l]; }

template <typename T>
__device__ __forceinline__ void batch_half(const BatchInst &I, const BPhase &ph, int tile) {
  const LevelT<T> &L = lview<T>(I.S, ph.level);
  const int slots = colour_slots(L.ni, L.nz);
  for (int r = 0; r < ph.grain; ++r) {
    const int t = (tile * ph.grain + r) * kBatchThreads + threadIdx.x;
    int i, j;
    if (t < slots && colour_node(t, L.ni, L.nz, ph.arg, i, j)) smooth_node<T>(L, i, j);
  }
}

template <typename T>
__device__ __forceinline__ void batch_restrict(const BatchInst &I, const BPhase &ph, int tile, unsigned char *buf) {
  const LevelT<T> &F = lview<T>(I.S, ph.level);
  const LevelT<T> &C = lview<T>(I.S, ph.level + 1);
  const int gx = (C.nr + 1 + kBatchRestrCX - 1) / kBatchRestrCX;
  for (int r = 0; r < ph.grain; ++r) {
    const int b = tile * ph.grain + r;
    // blocks past the grid find every coarse node out of range and only pass the barrier
    linres_restrict_tile<T, kBatchRestrCX, kBatchRestrCY>(F, C, (b % gx) * kBatchRestrCX, 1 + (b / gx) * kBatchRestrCY,
                                                          threadIdx.x, kBatchThreads, reinterpret_cast<T *>(buf));
    __syncthreads();
  }
}

template <typename T>
__device__ __forceinline__ void batch_prolong(const BatchInst &I, const BPhase &ph, int tile) {
  const LevelT<T> &F = lview<T>(I.S, ph.level);
  const LevelT<T> &C = lview<T>(I.S, ph.level + 1);
  const int n = F.ni * (F.nz - 1);
  for (int r = 0; r < ph.grain; ++r) {
    const int t = (tile * ph.grain + r) * kBatchThreads + threadIdx.x;
    if (t < n) prolong_node<T>(C, F, t % F.ni, t / F.ni + 1);
  }
}

template <typename T>
__device__ __forceinline__ void batch_zero(const LevelT<T> &L, const BPhase &ph, int tile) {
  const size_t n = (size_t)(L.nz + 1) * L.P;
  for (int r = 0; r < ph.grain; ++r) {
    const size_t t = (size_t)(tile * ph.grain + r) * kBatchThreads + threadIdx.x;
    if (t < n) { L.du[NE][t] = T(0); L.du[NP][t] = T(0); L.du[NV][t] = T(0); }
  }
}

__device__ void batch_tile(const BatchInst &I, const BPhase &ph, int tile, double *red, unsigned char *buf) {
  const LevelSet *S = I.S;
  const int tid = threadIdx.x;
  switch (ph.kind) {
    case BK_INJECT: {  // k_inject_levels: levels level .. arg from level - 1
      const Level &C1 = S->L[ph.level];
      const int l0 = ph.level - 1;
      const int gx = (C1.nr + 1 + 31) / 32, gy = (C1.nz + 1 + 7) / 8;
      for (int r = 0; r < ph.grain; ++r) {
        const int b = tile * ph.grain + r;
        if (b >= ph.nblocks) break;
        int lz, I_, J_;
        vb328(b, gx, gy, lz, I_, J_);
        const int l = ph.level + lz;
        const Level &C = S->L[l];
        if (I_ > C.nr || J_ > C.nz) continue;
        const int sh = l - l0;
        const size_t kc = (size_t)J_ * C.P + I_, kf = ((size_t)J_ << sh) * S->L[l0].P + ((size_t)I_ << sh);
#pragma unroll
        for (int q = 0; q < 3; ++q) S->sv[l].u[q][kc] = S->sv[l0].u[q][kf];
      }
      break;
    }
    case BK_INJECT1: {  // k_inject (state and sources) from level - 1 to level
      const Level &C = S->L[ph.level], &F = S->L[ph.level - 1];
      const StateView &cs = S->sv[ph.level], &fs = S->sv[ph.level - 1];
      const int gx = (C.nr + 1 + 31) / 32, gy = (C.nz + 1 + 7) / 8;
      for (int r = 0; r < ph.grain; ++r) {
        const int b = tile * ph.grain + r;
        if (b >= ph.nblocks) break;
        int lz, I_, J_;
        vb328(b, gx, gy, lz, I_, J_);
        if (I_ > C.nr || J_ > C.nz) continue;
        const size_t kc = (size_t)J_ * C.P + I_, kf = (size_t)(2 * J_) * F.P + 2 * I_;
#pragma unroll
        for (int q = 0; q < 3; ++q) cs.u[q][kc] = fs.u[q][kf];
        const_cast<double *>(cs.S[0])[kc] = fs.S[0][kf];
        const_cast<double *>(cs.S[1])[kc] = fs.S[1][kf];
      }
      break;
    }
    case BK_COEFL:
    case BK_COEF0: {  // k_coef_levels / k_coef: face coefficients of levels level .. arg
      const Level &La = S->L[ph.level];
      const int gx = (La.nr + 1 + 31) / 32, gy = (La.nz + 1 + 7) / 8;
      for (int r = 0; r < ph.grain; ++r) {
        const int b = tile * ph.grain + r;
        if (b >= ph.nblocks) break;
        int lz, i, j;
        vb328(b, gx, gy, lz, i, j);
        const int l = ph.level + lz;
        const Level &L = S->L[l];
        if (i > L.nr || j > L.nz) continue;
        coef_node(L, S->sv[l], I.tr, i, j);
      }
      break;
    }
    case BK_FACTORL: {  // k_factor_levels: levels level .. arg
      const Level &La = S->L[ph.level];
      const int gx = (La.nr + 1 + 31) / 32, gy = (La.nz + 1 + 7) / 8;
      for (int r = 0; r < ph.grain; ++r) {
        const int b = tile * ph.grain + r;
        if (b >= ph.nblocks) break;
        int lz, i, j;
        vb328(b, gx, gy, lz, i, j);
        const int l = ph.level + lz;
        const Level &L = S->L[l];
        if (i > L.nr || j > L.nz) continue;
        if (I.mixed) coef_to32_node(L, S->M[l], 1.0 / I.n0, (size_t)j * L.P + i);
        if (j >= 1 && j < L.nz && i < L.ni) factor_node(L, S->M[l], I.mixed, I.dt_inv, I.n0, i, j);
      }
      break;
    }
    case BK_CFACT: {  // k_coarse_factor_smem on the coarsest level
      double *sAB = reinterpret_cast<double *>(buf);
      double *srs = sAB + kSmemGJ * 2 * kSmemGJ, *scs = srs + kSmemGJ;
      int *sp = reinterpret_cast<int *>(scs + kSmemGJ);
      coarse_factor_smem_body(S->L[I.last], I.dt_inv, I.Minv, I.rs, I.cs, I.flag, sAB, srs, scs, sp);
      break;
    }
    case BK_ZERO64: batch_zero<double>(S->L[ph.level], ph, tile); break;
    case BK_ZERO32: batch_zero<float>(S->M[ph.level], ph, tile); break;
    case BK_NORM0:
    case BK_NORMC: {
      const Level &L = S->L[ph.level];
      if (I.mixed) {  // k_outer_residual: 32 x 8 blocks
        const int gx = (L.nr + 1 + 31) / 32, gy = (L.nz - 1 + 7) / 8;
        for (int r = 0; r < ph.grain; ++r) {
          const int b = tile * ph.grain + r;
          int lz, i, j;
          vb328(b, gx, gy, lz, i, j);
          double acc[3] = {0.0, 0.0, 0.0};
          if (b < ph.nblocks) outer_row(L, S->M[ph.level], 1.0 / I.n0, i, j + 1, acc);
          vblock_partial<3>(acc, 256, b < ph.nblocks, I.partials + (size_t)b * 3, red, 0);
        }
      } else {  // k_linres (f - J du into r): 32 x 2 blocks, four per round
        const int gx = (L.nr + 1 + 31) / 32;
        for (int r = 0; r < ph.grain; ++r) {
          const int b = (tile * ph.grain + r) * 4 + (tid >> 6);
          const int i = (b % gx) * 32 + (tid & 31), j = (b / gx) * 2 + ((tid >> 5) & 1) + 1;
          double acc[3] = {0, 0, 0};
          if (b < ph.nblocks && i < L.ni && j < L.nz) {
            const Triple<double> rr = linres_node<double>(L, i, j, L.du[NE], L.du[NP], L.du[NV], L.f[NE], L.f[NP],
                                                          L.f[NV], L.r[NE], L.r[NP], L.r[NV]);
            acc[0] = rr.e * rr.e; acc[1] = rr.p * rr.p; acc[2] = rr.V * rr.V;
          }
          vblock_partial<3>(acc, 64, b < ph.nblocks, I.partials + (size_t)b * 3, red, 0);
        }
      }
      break;
    }
    case BK_HALF64: batch_half<double>(I, ph, tile); break;
    case BK_HALF32: batch_half<float>(I, ph, tile); break;
    case BK_RESTR64: batch_restrict<double>(I, ph, tile, buf); break;
    case BK_RESTR32: batch_restrict<float>(I, ph, tile, buf); break;
    case BK_COARSE64:
      coarse_cycle_body<double>(*I.cs64[ph.level], tid, kBatchThreads, true, kBatchThreads, []() { __syncthreads(); });
      break;
    case BK_COARSE32:
      coarse_cycle_body<float>(*I.cs32[ph.level], tid, kBatchThreads, true, kBatchThreads, []() { __syncthreads(); });
      break;
    case BK_PROL64: batch_prolong<double>(I, ph, tile); break;
    case BK_PROL32: batch_prolong<float>(I, ph, tile); break;
    case BK_MIXUPD: {  // k_mixed_update
      const Level &L = S->L[ph.level];
      const LevelT<float> &M = S->M[ph.level];
      const int n = L.ni * (L.nz - 1);
      for (int r = 0; r < ph.grain; ++r) {
        const int t = (tile * ph.grain + r) * kBatchThreads + tid;
        if (t >= n) break;
        const size_t k = cidx(L.P, t % L.ni, t / L.ni + 1);
        L.du[NE][k] += I.n0 * (double)M.du[NE][k];
        L.du[NP][k] += I.n0 * (double)M.du[NP][k];
        L.du[NV][k] += (double)M.du[NV][k];
      }
      break;
    }
    case BK_UPDATE: {  // k_update: 32 x 8 blocks, maxima
      const Level &L = S->L[ph.level];
      const int gx = (L.nr + 1 + 31) / 32, gy = (L.nz - 1 + 7) / 8;
      for (int r = 0; r < ph.grain; ++r) {
        const int b = tile * ph.grain + r;
        int lz, i, j;
        vb328(b, gx, gy, lz, i, j);
        double acc[2] = {0.0, 0.0};
        if (b < ph.nblocks) update_row(L, S->sv[ph.level], i, j + 1, acc);
        vblock_partial<2>(acc, 256, b < ph.nblocks, I.partials + (size_t)b * 2, red, 1);
      }
      break;
    }
    case BK_RESID: {  // k_resid_coef: 32 x 2 blocks, four per round
      const Level &L = S->L[ph.level];
      const int gx = (L.nr + 1 + 31) / 32;
      const int wf = (ph.arg & RESID_WRITE_F) ? 1 : 0, st = (ph.arg & RESID_STEADY) ? 1 : 0;
      const double dti = (ph.arg & RESID_DT) ? I.dt_inv : 0.0;
      for (int r = 0; r < ph.grain; ++r) {
        const int b = (tile * ph.grain + r) * 4 + (tid >> 6);
        const int i = (b % gx) * 32 + (tid & 31), j = (b / gx) * 2 + ((tid >> 5) & 1) + 1;
        double acc[16];
        resid_row(L, S->sv[ph.level], dti, wf, st, nullptr, nullptr, nullptr, st ? I.fss[0] : nullptr,
                  st ? I.fss[1] : nullptr, st ? I.fss[2] : nullptr, b < ph.nblocks ? i : L.ni, j, acc);
        vblock_partial<16>(acc, 64, b < ph.nblocks, I.partials + (size_t)b * 16, red, 0);
      }
      break;
    }
    case BK_COPY: {  // the host's device-to-device copies of whole node arrays
      const Level &L = S->L[ph.level];
      const StateView &sv = S->sv[ph.level];
      const size_t n = (size_t)(L.nz + 1) * L.P;
      for (int r = 0; r < ph.grain; ++r) {
        const size_t t = (size_t)(tile * ph.grain + r) * kBatchThreads + tid;
        if (t >= n) break;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          if (ph.arg == COPY_TO_OLD) sv.uold[q][t] = sv.u[q][t];
          else if (ph.arg == COPY_FROM_OLD) sv.u[q][t] = sv.uold[q][t];
          else L.f[q][t] = I.fss[q][t];
        }
      }
      break;
    }
    case BK_PROLST: {  // k_prolong_state: level + 1 -> level, every node
      const Level &C = S->L[ph.level + 1], &F = S->L[ph.level];
      const StateView &cs = S->sv[ph.level + 1], &fs = S->sv[ph.level];
      const int n = (F.nr + 1) * (F.nz + 1);
      for (int r = 0; r < ph.grain; ++r) {
        const int t = (tile * ph.grain + r) * kBatchThreads + tid;
        if (t >= n) break;
        const int i = t % (F.nr + 1), j = t / (F.nr + 1);
        const size_t kf = (size_t)j * F.P + i;
        int J0, J1;
        double w0, w1;
        if (j & 1) { J0 = (j - 1) >> 1; J1 = J0 + 1; w1 = F.wz[j]; w0 = 1.0 - w1; }
        else { J0 = J1 = j >> 1; w0 = 1.0; w1 = 0.0; }
        int I0, I1;
        double v0, v1;
        if (i & 1) { I0 = (i - 1) >> 1; I1 = I0 + 1; v0 = v1 = 0.5; }
        else { I0 = I1 = i >> 1; v0 = 1.0; v1 = 0.0; }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const double *c = cs.u[q];
          const double a = v0 * c[(size_t)J0 * C.P + I0] + v1 * c[(size_t)J0 * C.P + I1];
          const double b = v0 * c[(size_t)J1 * C.P + I0] + v1 * c[(size_t)J1 * C.P + I1];
          fs.u[q][kf] = w0 * a + w1 * b;
        }
      }
      break;
    }
    case BK_DIRI: {  // k_dirichlet on level
      const Level &L = S->L[ph.level];
      const StateView &sv = S->sv[ph.level];
      const double Vc = I.m.Vc, Va = I.m.Va;
      const int n = (L.nr > L.nz ? L.nr : L.nz) + 1;
      for (int t = tid; t < n; t += kBatchThreads) {
        if (t <= L.nr) {
          const size_t k0 = t, k1 = (size_t)L.nz * L.P + t;
          sv.u[NE][k0] = 0.0; sv.u[NP][k0] = 0.0; sv.u[NV][k0] = Vc;
          sv.u[NE][k1] = 0.0; sv.u[NP][k1] = 0.0; sv.u[NV][k1] = Va;
        }
        if (L.ni == L.nr && t <= L.nz) {
          const size_t kw = (size_t)t * L.P + L.nr;
          sv.u[NE][kw] = 0.0; sv.u[NP][kw] = 0.0; sv.u[NV][kw] = Vc + (Va - Vc) * L.zf[t];
        }
      }
      break;
    }
    default: break;
  }
}

// ---- the steady solve of one discharge as a state machine (thread 0 of a finishing CTA) ----
// It follows the host driver (mg_solve_steady -> march -> step in mg_api.cu) statement by
// statement; std::max / std::min are (a < b ? b : a) / (b < a ? b : a), and the one expression
// with a product added to a sum is evaluated with rounded operations in the host's order.
enum { MS_INJECT = 0, MS_START, MS_BEGIN_USE, MS_BEGIN, MS_NEWTON, MS_RESTORE, MS_ACCSTART, MS_PROLONG };
constexpr int kMgOk = 0, kMgEnoconv = -3, kMgEreject = -4, kMgEnonfinite = -5;

__device__ __forceinline__ double hmax(double a, double b) { return (a < b) ? b : a; }
__device__ __forceinline__ double hmin(double a, double b) { return (b < a) ? b : a; }

__device__ __forceinline__ double ratio(double f2, double t2) {  // sqrt(f2) / sqrt(t2), as residual_norms
  const double fn = sqrt(f2), t = sqrt(t2);
  return fn == 0.0 ? 0.0 : (t > 0.0 ? fn / t : INFINITY);
}

__device__ __forceinline__ double steady_of_start(const BatchMarch &M) {
  double m = 0.0;
  for (int q = 0; q < 3; ++q) m = hmax(m, ratio(M.start_sums[6 + q], M.start_sums[9 + q]));
  return m;
}

__device__ __forceinline__ void count_coarse(BatchMarch &M) {
  M.coarse_steps = M.steps_accepted + M.steps_rejected;
  M.coarse_newton = M.newton_iterations;
  M.coarse_vcycles = M.vcycles;
}

__device__ int solve_end(BatchInst &I, int rc) {
  BatchMarch &M = I.m;
  if (!M.counted) count_coarse(M);
  M.rc = rc;
  M.t_done = global_ns();
  return -1;
}

__device__ int march_start(BatchInst &I, double dt_start) {
  BatchMarch &M = I.m;
  M.dt = dt_start;
  M.dt_prev = -1.0;
  M.coef_current = 0;
  M.r_start = 0.0;
  M.nstep = 0;
  M.stage = MS_START;
  return I.ent[M.lvl][E_START_COEF];
}

__device__ int step_begin(BatchInst &I) {
  BatchMarch &M = I.m;
  if (M.nstep >= M.max_steps) return solve_end(I, kMgEreject);
  M.step_tol = hmax(M.ntol, M.rel * M.r_start);
  M.r_step = -1.0;
  M.reason = kMgEnoconv;
  M.it = 0;
  for (int q = 0; q < 3; ++q) M.rho_steady[q] = -1.0;
  if (M.start_valid) {  // start_norms: the step's first residual from the start data
    const double *S = M.start_sums, c = 1.0 / M.dt;
    double t2[3];
    t2[0] = __dadd_rn(__dadd_rn(S[9], __dmul_rn(__dmul_rn(2.0, c), S[12])), __dmul_rn(__dmul_rn(c, c), S[13]));
    t2[1] = __dadd_rn(__dadd_rn(S[10], __dmul_rn(__dmul_rn(2.0, c), S[14])), __dmul_rn(__dmul_rn(c, c), S[15]));
    t2[2] = S[11];
    for (int q = 0; q < 3; ++q) {
      const double fn = sqrt(S[6 + q]), t = sqrt(t2[q]);
      M.tn[q] = t;
      M.rho[q] = fn == 0.0 ? 0.0 : (t > 0.0 ? fn / t : INFINITY);
    }
    M.stage = MS_BEGIN_USE;
    return I.ent[M.lvl][E_BEGIN_USE];
  }
  I.dt_inv = M.dt > 0 ? 1.0 / M.dt : 0.0;
  M.stage = MS_BEGIN;
  return I.ent[M.lvl][M.coef_current ? E_BEGIN : E_BEGIN_COEF];
}

__device__ int step_reject(BatchInst &I) {
  BatchMarch &M = I.m;
  M.newton_iterations += M.newton_out;
  M.last_newton = M.newton_out;
  M.stage = MS_RESTORE;
  return I.ent[M.lvl][E_RESTORE];
}

__device__ int march_end(BatchInst &I, int rc) {
  BatchMarch &M = I.m;
  if (rc != kMgOk) return solve_end(I, rc);
  const int l = M.lvl - 1;
  if (l < 0) return solve_end(I, kMgOk);
  if (l == 0) {
    count_coarse(M);
    M.counted = 1;
  }
  M.next_lvl = l;
  M.stage = MS_PROLONG;
  return I.ent[l][E_PROLONG];
}

__device__ int accepted2(BatchInst &I, double r) {
  BatchMarch &M = I.m;
  M.coef_current = 1;
  M.steady_rho = r;
  M.r_start = r;
  if (r <= M.tol) return march_end(I, kMgOk);
  M.dt_prev = M.dt;
  M.dt = hmin(M.dt * M.dt_growth, M.dt_max);
  ++M.nstep;
  return step_begin(I);
}

__device__ int step_accept(BatchInst &I) {
  BatchMarch &M = I.m;
  M.coef_current = 0;
  M.dt_last = M.dt;
  M.steps_accepted++;
  M.sim_time += M.dt;
  double r = M.r_step;
  if (r < 0.0) {
    if (!M.start_valid) {
      M.stage = MS_ACCSTART;
      return I.ent[M.lvl][E_START];
    }
    r = steady_of_start(M);
  }
  return accepted2(I, r);
}

// The Newton test at iteration M.it (rho, tn current): accept, reject or enter an iteration.
__device__ int newton_check(BatchInst &I) {
  BatchMarch &M = I.m;
  for (int q = 0; q < 3; ++q) M.srho[q] = M.rho[q];
  const double rmax = hmax(M.rho[0], hmax(M.rho[1], M.rho[2]));
  if (!(rmax == rmax) || isinf(rmax)) {
    M.reason = kMgEnonfinite;
    M.newton_out = M.it;
    return step_reject(I);
  }
  if (rmax <= M.step_tol) {
    if (M.it > 0) {
      M.r_step = hmax(M.rho_steady[0], hmax(M.rho_steady[1], M.rho_steady[2]));
      for (int q = 0; q < 16; ++q) M.start_sums[q] = M.cand[q];
      M.start_valid = 1;
    }
    M.newton_out = M.it;
    M.newton_iterations += M.it;
    M.last_newton = M.it;
    return step_accept(I);
  }
  if (M.it == M.max_newton) {
    M.newton_out = M.it;
    return step_reject(I);
  }
  M.start_valid = 0;
  const double eta = M.eta_adapt ? hmax(M.eta_p, hmin(0.1, 0.5 * M.step_tol / rmax)) : M.eta_p;
  I.eta = eta;
  for (int q = 0; q < 3; ++q) I.w[q] = M.tn[q] > 0.0 ? M.tn[q] : 1.0;
  I.dt_inv = M.dt > 0 ? 1.0 / M.dt : 0.0;
  M.stage = MS_NEWTON;
  return I.ent[M.lvl][E_NEWTON];
}

// A subprogram of discharge I has ended: the next program counter (-1: the solve has ended).
__device__ int batch_control(BatchInst &I) {
  BatchMarch &M = I.m;
  const double *o = I.dout;
  switch (M.stage) {
    case MS_INJECT:
      if (M.lvl < M.from) {
        ++M.lvl;
        return I.ent[M.lvl][E_INJECT];
      }
      return march_start(I, M.dt1);
    case MS_START:
      for (int q = 0; q < 16; ++q) M.start_sums[q] = o[q];
      M.start_valid = 1;
      M.coef_current = 1;
      M.r_start = steady_of_start(M);
      return step_begin(I);
    case MS_BEGIN:
      for (int q = 0; q < 3; ++q) {
        M.tn[q] = sqrt(o[3 + q]);
        M.rho[q] = ratio(o[q], o[3 + q]);
      }
      return newton_check(I);
    case MS_BEGIN_USE:
      return newton_check(I);
    case MS_NEWTON: {
      const SolveCtl *c = I.ctl;
      const bool ok = (c->r0 == 0.0) || (c->rel <= I.eta);
      M.vcycles += c->ncyc;
      if (!ok) { M.newton_out = M.it + 1; M.reason = kMgEnoconv; return step_reject(I); }
      if (o[17] != 0.0) { M.newton_out = M.it + 1; M.reason = kMgEnonfinite; return step_reject(I); }
      if (o[16] > M.limit) { M.newton_out = M.it + 1; M.reason = kMgEnoconv; return step_reject(I); }
      for (int q = 0; q < 3; ++q) {
        M.tn[q] = sqrt(o[3 + q]);
        M.rho[q] = ratio(o[q], o[3 + q]);
        M.rho_steady[q] = ratio(o[6 + q], o[9 + q]);
      }
      for (int q = 0; q < 16; ++q) M.cand[q] = o[q];
      ++M.it;
      return newton_check(I);
    }
    case MS_RESTORE:
      M.coef_current = 0;
      M.dt_last = M.dt;
      M.steps_rejected++;
      if (M.dt_prev > 0.0 && M.dt > M.dt_prev) {
        M.dt = M.dt_prev;
      } else {
        M.dt *= 0.5;
        if (M.dt_prev > 0.0) M.dt_prev = hmin(M.dt_prev, M.dt);
      }
      ++M.nstep;
      return step_begin(I);
    case MS_ACCSTART:
      for (int q = 0; q < 16; ++q) M.start_sums[q] = o[q];
      M.start_valid = 1;
      return accepted2(I, steady_of_start(M));
    case MS_PROLONG:
      M.lvl = M.next_lvl;
      return march_start(I, M.dt_max);
    default:
      return solve_end(I, kMgEreject);
  }
}

// The finisher of a phase (every thread of its CTA): fold the phase's reduction; thread 0 then
// takes the V-cycle loop's stopping test or the state machine's next step and publishes the
// next phase.
// Returns (thread 0) the program counter of the new phase whose first work item this CTA keeps,
// or -1 when the solve has ended.
__device__ int batch_finish(BatchInst &I, const BPhase &ph, int pc, unsigned seq, BatchHead *head, double *red) {
  switch (ph.kind) {
    case BK_NORM0:
    case BK_NORMC: fold_partials<3>(I.partials, ph.nblocks, I.mixed ? 256 : 64, I.dout, red, 0); break;
    case BK_UPDATE: fold_partials<2>(I.partials, ph.nblocks, 256, I.dout + 16, red, 1); break;
    case BK_RESID: fold_partials<16>(I.partials, ph.nblocks, 64, I.dout, red, 0); break;
    default: break;
  }
  if (threadIdx.x != 0) return -1;
  int next = pc + 1;
  SolveCtl *c = I.ctl;
  if (ph.kind == BK_NORM0) {  // k_solve_init
    for (int q = 0; q < 3; ++q) c->w[q] = I.w[q];
    c->eta = I.eta;
    c->max_cycles = I.max_cycles;
    const double r0 = weighted_norm(c, I.dout);
    c->r0 = r0;
    c->ncyc = 0;
    c->rel = r0 > 0.0 ? 1.0 : 0.0;
    c->hist[0] = c->rel;
    const bool go = r0 > 0.0 && isfinite(r0) && c->rel > c->eta && c->max_cycles > 0;
    next = go ? I.ent[ph.level][E_NLOOP] : I.ent[ph.level][E_NUPD];
  } else if (ph.kind == BK_NORMC) {  // k_solve_check
    const double rel = weighted_norm(c, I.dout) / c->r0;
    const int n = c->ncyc + 1;
    c->ncyc = n;
    c->rel = rel;
    if (n < kMaxHist) c->hist[n] = rel;
    const bool go = isfinite(rel) && rel > c->eta && n < c->max_cycles;
    next = go ? I.ent[ph.level][E_NLOOP] : I.ent[ph.level][E_NUPD];
  }
  if (I.prog[next].kind == BK_RET) next = batch_control(I);
  const bool ended = next < 0;
  const unsigned ns = seq + 1;
  const int nt = ended ? 0 : I.prog[next].ntiles;
  I.ring[ns & 3] = ring_entry(ns, ended ? 0 : next, nt);
  I.done = 0u;
  // the finisher keeps the new phase's first work item for itself (count 1)
  atom_exch_release64(&I.claim, ((unsigned long long)ns << 32) | (nt > 0 ? 1u : 0u));
  atomicAdd(&head->progress, 1u);
  if (ended) atomicAdd(&head->ndone, 1);
  return nt > 0 ? next : -1;
}

__global__ void __launch_bounds__(kBatchThreads, 3) k_batch(BatchHead *head, BatchInst *inst) {
  extern __shared__ __align__(16) unsigned char bsm[];
  double *red = reinterpret_cast<double *>(bsm);
  unsigned char *buf = bsm + kBatchShRed;
  __shared__ int s_k, s_pc, s_tile, s_last, s_exit, s_keep;
  __shared__ unsigned s_seq;
  const int n = head->n;
  if (threadIdx.x == 0) {
    atomicMin(&head->t0, global_ns());
    s_keep = 0;
  }
  int own = blockIdx.x % (n > 0 ? n : 1);   // the discharge this CTA worked on last
  // whether discharge k has an unclaimed work item (a hint: the claim decides)
  auto open = [&](int k) {
    const BatchInst &I = inst[k];
    const unsigned long long w = ld_vol64(&I.claim);
    const unsigned seq = (unsigned)(w >> 32), cnt = (unsigned)w;
    const unsigned long long e = ld_vol64(&I.ring[seq & 3]);
    return (unsigned)(e >> 32) == seq && cnt < ring_ntiles(e);
  };
  for (;;) {
    if (threadIdx.x < 32 && !s_keep) {
      // warp 0 looks for work: first the discharge it worked on last (the next phase it may just
      // have published), then every discharge at once, one per lane, the first open one in index
      // order (largest discharges first: the longest chains of phases); lane 0 claims it
      const int lane = threadIdx.x;
      unsigned pause = 32;
      unsigned seen = *reinterpret_cast<volatile unsigned *>(&head->progress);
      unsigned long long idle0 = global_ns();
      int exit_now = 0;
      for (unsigned spin = 0;; ++spin) {
        int cand = (lane == 0 && open(own)) ? own : -1;
        cand = __shfl_sync(0xffffffffu, cand, 0);
        for (int base = 0; base < n && cand < 0; base += 32) {
          const int k = base + lane;
          const unsigned m = __ballot_sync(0xffffffffu, k < n && open(k));
          if (m) cand = base + __ffs(m) - 1;
        }
        int got = 0;
        if (cand >= 0 && lane == 0) {
          BatchInst &I = inst[cand];
          const unsigned long long o = atom_add_acqrel64(&I.claim, 1ull);
          const unsigned s2 = (unsigned)(o >> 32), c2 = (unsigned)o;
          const unsigned long long e2 = ld_vol64(&I.ring[s2 & 3]);
          if ((unsigned)(e2 >> 32) == s2 && c2 < ring_ntiles(e2)) {
            s_k = cand; s_pc = ring_pc(e2); s_tile = (int)c2; s_seq = s2;
            got = 1;
          }
        }
        got = __shfl_sync(0xffffffffu, got, 0);
        if (got) {
          own = cand;
          break;
        }
        if (lane == 0) {
          if (*reinterpret_cast<volatile unsigned *>(&head->err) != 0 ||
              *reinterpret_cast<volatile int *>(&head->ndone) >= n) {
            exit_now = 1;
          } else if ((spin & 15) == 15) {
            const unsigned now_seen = *reinterpret_cast<volatile unsigned *>(&head->progress);
            const unsigned long long now = global_ns();
            if (now_seen != seen) {
              seen = now_seen;
              idle0 = now;
            } else if (now - idle0 > kBatchIdleNs) {
              atomicExch(&head->err, 1u);
              exit_now = 1;
            }
          }
        }
        exit_now = __shfl_sync(0xffffffffu, exit_now, 0);
        if (exit_now) break;
        if (cand >= 0) continue;  // lost the race for that item: look again at once
        __nanosleep(pause);
        if (pause < 512) pause <<= 1;
      }
      if (lane == 0) s_exit = exit_now;
    }
    __syncthreads();
    if (s_exit) return;
    const int k = s_k, pc = s_pc, tile = s_tile;
    const unsigned seq = s_seq;
    BatchInst &I = inst[k];
    const BPhase ph = I.prog[pc];
    batch_tile(I, ph, tile, red, buf);
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned d = atom_add_acqrel32(&I.done, 1u);
      s_last = (d + 1 == (unsigned)ph.ntiles);
      s_keep = 0;
    }
    __syncthreads();
    if (s_last) {
      const int next = batch_finish(I, ph, pc, seq, head, red);
      if (threadIdx.x == 0 && next >= 0) {  // this CTA runs the new phase's first work item
        s_k = k; s_pc = next; s_tile = 0; s_seq = seq + 1;
        s_keep = 1;
        s_exit = 0;
      }
    }
    __syncthreads();
  }
}

int batch_grid() {
  static std::once_flag once;
  static int cached = 0;
  std::call_once(once, []() {
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch, kBatchThreads, kBatchSmem) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    cached = sms * occ;
  });
  return cached;
}

cudaError_t launch_batch(BatchHead *head, BatchInst *inst, int grid, cudaStream_t st) {
  k_batch<<<grid, kBatchThreads, kBatchSmem, st>>>(head, inst);
  count_launch();
  return cudaGetLastError();
}

}  // namespace mgk

// ==========================================================================================
// Allocation-free residual entry point (declared in include/mg.h as mg_residual_noalloc).
//
// Some callers cannot allocate device memory: code that runs inside another framework's
// memory pool or a real-time loop where cudaMalloc is forbidden or would synchronise the
// device, and plug-ins that may only use the buffers their host hands them.  For them this
// entry point evaluates the same residual rows and norms as mg_residual (up to rounding: it
// evaluates every face directly with k_residual instead of through stored face coefficients)
// on caller-owned input and output arrays, and keeps its own scratch (geometry,
// transport table, block partial sums, reduction counter and results) in the file-scope
// device array below.  Every GPU that loads this library holds that array until the process
// exits.  All calls share it and it keeps the last call's contents: calls that overlap on the
// GPU (different streams, threads or devices' streams racing on one device) race on it.
#include <mutex>

#include "../../include/mg.h"

namespace {

constexpr int kNoallocMaxN = 1024;                       // largest N_r, N_z accepted
constexpr int kNoallocGeo = kNoallocMaxN + 2;            // length of each geometry vector
constexpr int kNoallocTableRows = 64;
constexpr int kNoallocBlocks = ((kNoallocMaxN + 1 + 31) / 32) * ((kNoallocMaxN - 1 + 7) / 8);
// layout (doubles): results [0, 8) | counter [8, 16) | dz | dzc | volr | table | partials
constexpr size_t kOffOut = 0, kOffCounter = 8, kOffDz = 16;
constexpr size_t kOffDzc = kOffDz + kNoallocGeo, kOffVolr = kOffDzc + kNoallocGeo;
constexpr size_t kOffTable = kOffVolr + kNoallocGeo;
constexpr size_t kOffPartials = kOffTable + 5 * kNoallocTableRows;
constexpr size_t kNoallocDoubles = kOffPartials + 6 * (size_t)kNoallocBlocks;  // ~232 KB

}  // namespace

static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

namespace {

std::mutex g_noalloc_mu;
double *g_noalloc_addr[128];  // device address of g_noalloc_scratch, per device ordinal

// Device address of the scratch array on the current device, looked up once per device
// (with that device current).  In host code the array's name is only a host-side stand-in.
cudaError_t noalloc_scratch(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = static_cast<double *>(p);
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int mg_residual_noalloc(const mg_grid *g, const mg_params *p, const double *ne, const double *np,
                                   const double *V, const double *ne_old, const double *np_old, const double *V_old,
                                   const double *S_e, const double *S_p, double dt, double *F_ne, double *F_np,
                                   double *F_V, double rho[3], void *stream) {
  using namespace mgk;
  if (!g || !p || !g->z || !ne || !np || !V || !S_e || !S_p || !rho) return MG_EINVAL;
  const int nr = g->nr, nz = g->nz;
  auto pow2 = [](int x) { return x >= 2 && (x & (x - 1)) == 0; };
  if (!pow2(nr) || !pow2(nz) || nr > kNoallocMaxN || nz > kNoallocMaxN || !(g->R > 0.0)) return MG_EINVAL;
  if (dt > 0.0 && (!ne_old || !np_old || !V_old)) return MG_EINVAL;
  if ((F_ne || F_np || F_V) && !(F_ne && F_np && F_V)) return MG_EINVAL;
  if (!(p->pressure_factor > 0.0) || !(p->D_e > 0.0) || !(p->D_p > 0.0)) return MG_EINVAL;
  if (p->table && (p->table_rows < 2 || p->table_rows > kNoallocTableRows)) return MG_EINVAL;
  if (p->wall_dirichlet) return MG_EINVAL;  // wall rows are those of the zero-flux wall
  for (int j = 0; j < nz; ++j)
    if (!(g->z[j + 1] > g->z[j])) return MG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  double *base = nullptr;
  if (noalloc_scratch(&base) != cudaSuccess) return MG_ECUDA;

  // geometry of the finite-volume rows (same formulas as the state-based path), built on the
  // host in fixed-size buffers and copied into the scratch array
  double geo[3][kNoallocGeo];
  const double dr = g->R / nr;
  for (int q = 0; q < 3; ++q)
    for (int k = 0; k < kNoallocGeo; ++k) geo[q][k] = 0.0;
  for (int j = 0; j < nz; ++j) geo[0][j] = g->z[j + 1] - g->z[j];
  for (int j = 1; j < nz; ++j) geo[1][j] = 0.5 * (geo[0][j - 1] + geo[0][j]);
  for (int i = 0; i <= nr; ++i) geo[2][i] = i * dr * dr;
  geo[2][0] = dr * dr / 8.0;
  geo[2][nr] = (nr - 0.25) * dr * dr / 2.0;
  if (cudaMemcpyAsync(base + kOffDz, geo, sizeof(geo), cudaMemcpyHostToDevice, st) != cudaSuccess) return MG_ECUDA;
  if (p->table && cudaMemcpyAsync(base + kOffTable, p->table, sizeof(double) * 5 * p->table_rows,
                                  cudaMemcpyHostToDevice, st) != cudaSuccess)
    return MG_ECUDA;
  // the reduction counter must start at zero (an earlier call that failed may have left it set)
  if (cudaMemsetAsync(base + kOffCounter, 0, sizeof(double), st) != cudaSuccess) return MG_ECUDA;

  Level L = Level();
  L.nr = nr; L.nz = nz; L.P = nr + 1;  // caller arrays are dense rows of nr + 1 nodes
  L.ni = nr + 1;
  L.dr = dr;
  L.dz = base + kOffDz; L.dzc = base + kOffDzc; L.volr = base + kOffVolr;
  StateView sv;
  sv.u[NE] = const_cast<double *>(ne); sv.u[NP] = const_cast<double *>(np); sv.u[NV] = const_cast<double *>(V);
  sv.uold[NE] = const_cast<double *>(ne_old); sv.uold[NP] = const_cast<double *>(np_old);
  sv.uold[NV] = const_cast<double *>(V_old);
  sv.S[0] = S_e; sv.S[1] = S_p;
  Transport tr;
  tr.mu_e = p->mu_e / p->pressure_factor; tr.D_e = p->D_e / p->pressure_factor;
  tr.mu_p = p->mu_p / p->pressure_factor; tr.D_p = p->D_p / p->pressure_factor;
  tr.inv_pf = 1.0 / p->pressure_factor;
  tr.table = p->table ? base + kOffTable : nullptr;
  tr.rows = p->table ? p->table_rows : 0;
  tr.inv_dE = nullptr;
  double *Fo[3] = {F_ne, F_np, F_V};
  if (launch_residual(L, sv, tr, dt, false, F_ne ? Fo : nullptr, base + kOffPartials,
                      reinterpret_cast<unsigned *>(base + kOffCounter), base + kOffOut, st) != cudaSuccess)
    return MG_ECUDA;
  double out6[6];
  if (cudaMemcpyAsync(out6, base + kOffOut, sizeof(out6), cudaMemcpyDeviceToHost, st) != cudaSuccess) return MG_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MG_ECUDA;
  for (int q = 0; q < 3; ++q) {
    const double fn = sqrt(out6[q]), t = sqrt(out6[3 + q]);
    rho[q] = fn == 0.0 ? 0.0 : (t > 0.0 ? fn / t : INFINITY);
  }
  return MG_OK;
}
