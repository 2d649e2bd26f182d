// Host side of the C ABI declared in include/mg.h: state and workspace layout, the multigrid
// V-cycle schedule, Newton-Raphson, the Delta-t ramp and the coarse-to-fine continuation
// (Ristivojevic & Petrovic, arXiv:0811.4446, Sec. 2).  All arithmetic on the solution runs in
// the kernels of mg_kernels.cu; the host only sequences launches and reads back norms.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <chrono>
#include <new>
#include <thread>
#include <string>
#include <vector>

#include "../../include/mg.h"
#include "../../include/mg_debug.h"
#include "mg_impl.cuh"

using namespace mgk;

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxLevels = 16;
constexpr int kMaxCoarse = 3 * 9 * 9;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }
bool pow2(int x) { return x >= 2 && (x & (x - 1)) == 0; }

// Host-side record of one level: dimensions and device pointers.
struct LevelBuf {
  int nr, nz, P;
  size_t nodes;
  Level L;               // FP64 view (geometry + MG work arrays)
  LevelT<float> M;       // FP32 view (mixed form only)
  StateView sv;          // FP64 nonlinear state on this level
  double *geo;           // device geometry block
  float *geo32;
  double *ubak[3];       // copy of the state (fallback of the learned-guess solve)
  int sbx = 32, sby = 2;         // half-sweep launch shape, FP64 view (autotuned)
  int sbx32 = 32, sby32 = 2;     // half-sweep launch shape, FP32 view (autotuned)
  int sw = 1, sw32 = 1;          // fused-sweep tile shape index, FP64 / FP32 (autotuned)
  int fuse = 0, fuse32 = 1;      // fused sweep on this level (FP64: off, see mg_autotune; FP32: autotuned)
  int nu1 = -1, nu2 = -1;        // sweeps set by mg_set_level_sweeps (-1: the parameters' rule)
};

}  // namespace

struct mg_state {
  mg_params prm;
  std::vector<double> table_h;
  int nr, nz;
  double R;
  std::vector<double> z;
  int nlev;
  LevelBuf lv[kMaxLevels];
  Transport tr;
  cudaStream_t stream;
  void *ws;
  size_t ws_bytes;
  bool owns_ws;
  // scratch
  double *partials;
  size_t partials_cap;   // doubles
  unsigned *counter;
  double *dout;          // device outputs of reductions (24 doubles)
  double *hout;          // pinned host mirror (24 doubles)
  double *M, *Minv, *rs, *cs;
  double *fj_f[3], *fj_d[3];  // full-Jacobian Newton: saved right-hand side and accumulated step
  double *fss[3];             // -F of the steady rows at the current state (a march step's first f)
  double start_sums[16];      // the residual sums of that launch (see k_resid_coef)
  bool start_valid = false;   // fss and start_sums describe the current state of the march level
  double *line_scr;           // z-line smoother: 12 planes of (nz + 1) x (nr + 2) / 2 of the finest level
  int *flag;
  double *table_d;
  mg_stats stats;
  std::string err;
  // kernel timing (mg_profile_begin / mg_profile_end)
  int prof_kernel = 0, prof_level = -1, prof_n = 0;
  std::vector<cudaEvent_t> prof_ev;
  // device-side linear solves: one instantiated graph per root level
  cudaStream_t cap_stream = nullptr;
  SolveCtl *ctl = nullptr, *hctl = nullptr;
  cudaGraphExec_t vexec[kMaxLevels] = {};
  int vprefix[kMaxLevels] = {}, vbody[kMaxLevels] = {};
  // persistent coarse-cycle kernel: levels cc_from .. nlev-1 in one cluster launch
  int cc_from = -1;
  CoarseSet<double> *cset64 = nullptr;
  CoarseSet<float> *cset32 = nullptr;
  size_t cc_smem64 = 0, cc_smem32 = 0;  // shared memory of the single-CTA form (0: global-memory form)
  LevelSet *lset = nullptr;   // device copy of every level's views (multi-level set-up kernels)
  // batched form: the device program of the steady solve (built on first use)
  BPhase *bprog = nullptr;
  int bent[kMaxLevelSet][E_N] = {};          // its subprogram entries per level
  int bgrain = 4;                            // thread-block rounds per work item
  int bcoarse_n = 16;                        // levels with at most this many intervals per side run
                                             // in the single-CTA coarse phase of the V-cycle
  int host_prog_ntiles0 = 0;                 // work items of the program's first phase
  CoarseSet<double> *bcs64[kMaxLevels] = {}; // device coarse sets of the batched program by start level
  CoarseSet<float> *bcs32[kMaxLevels] = {};
};

namespace {

int fail(mg_state *s, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (s) s->err = buf;
  return code;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail(s, MG_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Level dimensions of the hierarchy.
int plan_levels(int nr, int nz, int coarsest, int *lnr, int *lnz) {
  int n = 0;
  lnr[n] = nr; lnz[n] = nz; ++n;
  while (n < kMaxLevels && std::min(lnr[n - 1], lnz[n - 1]) > coarsest && lnr[n - 1] % 2 == 0 && lnz[n - 1] % 2 == 0) {
    lnr[n] = lnr[n - 1] / 2; lnz[n] = lnz[n - 1] / 2; ++n;
  }
  return n;
}

int pitch_of(int nr) { return ((nr + 1) + 3) & ~3; }

// Workspace layout: computed twice, once to size it and once to carve it.
struct Carver {
  char *base;
  size_t off;
  template <typename T>
  T *take(size_t count) {
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += align_up(count * sizeof(T));
    return p;
  }
};

constexpr int kFieldsPerLevel = 48;  // u 3, uold 3, S 2, cr 6, cz 6, du 3, f 3, r 3, gR gZ Ak 3, fac 7, dia 3, ubak 3, du2 3
constexpr int kGeoPerLevel = 6;      // dz, dzc, volr, wz, 1/dz, z fraction (each up to max(nr, nz) + 1)

// blocks of the largest reduction launch (32 x 2 threads per block)
size_t max_blocks(int nr, int nz) { return (size_t)((nr + 1 + 31) / 32) * ((nz + 1 + 1) / 2); }

constexpr int kFields32PerLevel = 37;  // cr 6, cz 6, du 3, f 3, r 3, gR gZ Ak 3, fac 7, dia 3, du2 3

void carve(Carver &c, mg_state *s, int nlev, const int *lnr, const int *lnz, int table_rows, bool mixed,
           bool line) {
  for (int l = 0; l < nlev; ++l) {
    LevelBuf &b = s->lv[l];
    b.nr = lnr[l]; b.nz = lnz[l]; b.P = pitch_of(lnr[l]);
    b.nodes = (size_t)(b.nz + 1) * b.P;
    const int glen = std::max(b.nr, b.nz) + 2;
    b.geo = c.take<double>((size_t)kGeoPerLevel * glen);
    double *f[kFieldsPerLevel];
    for (int q = 0; q < kFieldsPerLevel; ++q) f[q] = c.take<double>(b.nodes);
    int q = 0;
    for (int a = 0; a < 3; ++a) b.sv.u[a] = f[q++];
    for (int a = 0; a < 3; ++a) b.sv.uold[a] = f[q++];
    for (int a = 0; a < 2; ++a) b.sv.S[a] = f[q++];
    for (int a = 0; a < NCOEF; ++a) b.L.cr[a] = f[q++];
    for (int a = 0; a < NCOEF; ++a) b.L.cz[a] = f[q++];
    for (int a = 0; a < 3; ++a) b.L.du[a] = f[q++];
    for (int a = 0; a < 3; ++a) b.L.f[a] = f[q++];
    for (int a = 0; a < 3; ++a) b.L.r[a] = f[q++];
    b.L.gR = f[q++]; b.L.gZ = f[q++]; b.L.Ak = f[q++];
    for (int a = 0; a < NFAC; ++a) b.L.fac[a] = f[q++];
    for (int a = 0; a < NDIA; ++a) b.L.dia[a] = f[q++];
    for (int a = 0; a < 3; ++a) b.ubak[a] = f[q++];
    for (int a = 0; a < 3; ++a) b.L.du2[a] = f[q++];
    b.L.nr = b.nr; b.L.nz = b.nz; b.L.P = b.P;
    if (b.geo) {
      b.L.dz = b.geo;
      b.L.dzc = b.geo + glen;
      b.L.volr = b.geo + 2 * glen;
      b.L.wz = b.geo + 3 * glen;
      b.L.idz = b.geo + 4 * glen;
      b.L.zf = b.geo + 5 * glen;
    }
    b.M = LevelT<float>();
    b.geo32 = nullptr;
    if (mixed) {
      b.geo32 = c.take<float>((size_t)kGeoPerLevel * glen);
      float *g[kFields32PerLevel];
      for (int q2 = 0; q2 < kFields32PerLevel; ++q2) g[q2] = c.take<float>(b.nodes);
      int w = 0;
      for (int a = 0; a < NCOEF; ++a) b.M.cr[a] = g[w++];
      for (int a = 0; a < NCOEF; ++a) b.M.cz[a] = g[w++];
      for (int a = 0; a < 3; ++a) b.M.du[a] = g[w++];
      for (int a = 0; a < 3; ++a) b.M.f[a] = g[w++];
      for (int a = 0; a < 3; ++a) b.M.r[a] = g[w++];
      b.M.gR = g[w++]; b.M.gZ = g[w++]; b.M.Ak = g[w++];
      for (int a = 0; a < NFAC; ++a) b.M.fac[a] = g[w++];
      for (int a = 0; a < NDIA; ++a) b.M.dia[a] = g[w++];
      for (int a = 0; a < 3; ++a) b.M.du2[a] = g[w++];
      b.M.nr = b.nr; b.M.nz = b.nz; b.M.P = b.P;
      if (b.geo32) {
        b.M.dz = b.geo32;
        b.M.dzc = b.geo32 + glen;
        b.M.volr = b.geo32 + 2 * glen;
        b.M.wz = b.geo32 + 3 * glen;
        b.M.idz = b.geo32 + 4 * glen;
        b.M.zf = b.geo32 + 5 * glen;
      }
    }
  }
  s->partials_cap = 16 * max_blocks(lnr[0], lnz[0]) + 64;
  s->partials = c.take<double>(s->partials_cap);
  s->counter = c.take<unsigned>(4);
  s->dout = c.take<double>(24);
  s->M = c.take<double>((size_t)kMaxCoarse * kMaxCoarse);
  s->Minv = c.take<double>((size_t)kMaxCoarse * kMaxCoarse);
  s->rs = c.take<double>(kMaxCoarse);
  s->cs = c.take<double>(kMaxCoarse);
  s->flag = c.take<int>(4);
  s->ctl = c.take<SolveCtl>(1);
  s->cset64 = c.take<CoarseSet<double>>(1);
  s->cset32 = c.take<CoarseSet<float>>(1);
  s->table_d = table_rows > 0 ? c.take<double>((size_t)table_rows * 6) : nullptr;  // rows x 5, then 1/dE
  s->lset = c.take<LevelSet>(1);
  {
    const size_t n0 = (size_t)(lnz[0] + 1) * pitch_of(lnr[0]);
    for (int q = 0; q < 3; ++q) { s->fj_f[q] = c.take<double>(n0); s->fj_d[q] = c.take<double>(n0); }
    for (int q = 0; q < 3; ++q) s->fss[q] = c.take<double>(n0);
  }
  s->line_scr = line ? c.take<double>((size_t)12 * (lnz[0] + 1) * ((lnr[0] + 2) / 2)) : nullptr;
}

// Geometry of one level (finite-volume control volumes of eqs. 12-13, per radian).
void host_geometry(const std::vector<double> &zl, int nr, double R, std::vector<double> &out, int glen) {
  const int nz = (int)zl.size() - 1;
  out.assign((size_t)kGeoPerLevel * glen, 0.0);
  double *dz = out.data(), *dzc = dz + glen, *volr = dz + 2 * glen, *wz = dz + 3 * glen, *idz = dz + 4 * glen,
         *zf = dz + 5 * glen;
  const double dr = R / nr;
  for (int j = 0; j < nz; ++j) dz[j] = zl[j + 1] - zl[j];
  for (int j = 0; j < nz; ++j) idz[j] = 1.0 / dz[j];
  for (int j = 0; j <= nz; ++j) zf[j] = (zl[j] - zl[0]) / (zl[nz] - zl[0]);
  for (int j = 1; j < nz; ++j) dzc[j] = 0.5 * (dz[j - 1] + dz[j]);
  for (int i = 0; i <= nr; ++i) volr[i] = i * dr * dr;
  volr[0] = dr * dr / 8.0;
  volr[nr] = (nr - 0.25) * dr * dr / 2.0;
  for (int j = 1; j < nz; j += 2) wz[j] = (zl[j] - zl[j - 1]) / (zl[j + 1] - zl[j - 1]);
}

cudaMemcpyKind kind_in(int where) { return where == MG_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }
cudaMemcpyKind kind_out(int where) { return where == MG_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }

// Copy rows [j0, j1] of a dense (nz+1) x (nr+1) caller array into a pitched level array.
int copy_in(mg_state *s, const LevelBuf &b, double *dst, const double *src, int where, int j0, int j1) {
  const size_t w = (size_t)(b.nr + 1) * sizeof(double);
  CK(cudaMemcpy2DAsync(dst + (size_t)j0 * b.P, b.P * sizeof(double), src + (size_t)j0 * (b.nr + 1), w, w,
                       j1 - j0 + 1, kind_in(where), s->stream));
  return MG_OK;
}

int copy_out(mg_state *s, const LevelBuf &b, double *dst, const double *src, int where) {
  const size_t w = (size_t)(b.nr + 1) * sizeof(double);
  CK(cudaMemcpy2DAsync(dst, w, src, b.P * sizeof(double), w, b.nz + 1, kind_out(where), s->stream));
  return MG_OK;
}

bool mixed(const mg_state *s) { return s->prm.precision == MG_MIXED; }

int sync_read(mg_state *s, int n) {
  CK(cudaMemcpyAsync(s->hout, s->dout, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return MG_OK;
}

constexpr int kProfMax = 16384;

// Record a timing event pair around one launch when (kernel, level) is being profiled.
struct ProfScope {
  mg_state *s;
  bool on;
  ProfScope(mg_state *s_, int kernel, int level) : s(s_), on(false) {
    if (s->prof_kernel == kernel && s->prof_level == level && s->prof_n < kProfMax) {
      on = true;
      cudaEventRecord(s->prof_ev[2 * s->prof_n], s->stream);
    }
  }
  ~ProfScope() {
    if (on) {
      cudaEventRecord(s->prof_ev[2 * s->prof_n + 1], s->stream);
      s->prof_n++;
    }
  }
};

// ---------------------------------------------------------------- building blocks
// Nonlinear residual on root level l0: launches only.  with_coef: the face coefficients are
// (re)computed at the current state first; callers pass false only right after a residual at
// the same state (the coefficients are also the Jacobian's, reused by build_hierarchy).  The six
// sums of squares land in dout[0..5]; with steady_too those of the steady rows (no
// time-derivative terms) in dout[6..11] as well.
int residual_launch(mg_state *s, int l0, double dt, bool write_f, double *Fout[3], bool with_coef,
                    bool steady_too = false) {
  LevelBuf &b = s->lv[l0];
  ProfScope ps(s, MG_PROF_RESIDUAL, l0);
  if (with_coef) CK(launch_coef(b.L, b.sv, s->tr, s->stream));
  CK(launch_resid_coef(b.L, b.sv, dt, write_f, steady_too, Fout, steady_too ? s->fss : nullptr, s->partials,
                       s->counter, s->dout, s->stream));
  return MG_OK;
}

// rho[3] and the term norms tn[3] from the sums read back into hout[0..5]
void residual_norms(const mg_state *s, double rho[3], double tn[3]) {
  for (int q = 0; q < 3; ++q) {
    const double fn = std::sqrt(s->hout[q]), t = std::sqrt(s->hout[3 + q]);
    if (tn) tn[q] = t;
    if (rho) rho[q] = fn == 0.0 ? 0.0 : (t > 0.0 ? fn / t : INFINITY);
  }
}

// Nonlinear residual on root level l0; rho[3] and the term norms tn[3]; f = -F written if write_f.
int residual(mg_state *s, int l0, double dt, bool write_f, double *Fout[3], double rho[3], double tn[3],
             bool with_coef = true) {
  int rc = residual_launch(s, l0, dt, write_f, Fout, with_coef);
  if (rc || (rc = sync_read(s, 6))) return rc;
  residual_norms(s, rho, tn);
  return MG_OK;
}

// Start data of a march step at the current state of level l0 (the steady rows' -F in fss and
// the sums of k_resid_coef in start_sums), from one residual launch; with_coef as in
// residual_launch.
int start_data(mg_state *s, int l0, bool with_coef) {
  int rc = residual_launch(s, l0, 0.0, false, nullptr, with_coef, true);
  if (rc || (rc = sync_read(s, 16))) return rc;
  for (int q = 0; q < 16; ++q) s->start_sums[q] = s->hout[q];
  s->start_valid = true;
  return MG_OK;
}

// rho[3] and tn[3] of a step of length dt that starts from the state start_sums describe (its F
// is the steady one; its e and p term norms gain the time terms t / dt).
void start_norms(const mg_state *s, double dt, double rho[3], double tn[3]) {
  const double *S = s->start_sums, c = 1.0 / dt;
  const double t2[3] = {S[9] + 2.0 * c * S[12] + c * c * S[13], S[10] + 2.0 * c * S[14] + c * c * S[15], S[11]};
  for (int q = 0; q < 3; ++q) {
    const double fn = std::sqrt(S[6 + q]), t = std::sqrt(t2[q]);
    tn[q] = t;
    rho[q] = fn == 0.0 ? 0.0 : (t > 0.0 ? fn / t : INFINITY);
  }
}

// Coefficients on levels l0..nlev-1 at the state of l0 injected downward; coarsest inverse.
// The face coefficients of level l0 itself come from residual() at the same state, which every
// caller runs first.  All coarser levels are treated by one launch per phase (their kernels are
// latency-bound one by one).
int build_hierarchy(mg_state *s, int l0, double dt) {
  const int last = s->nlev - 1;
  {
    ProfScope ps(s, MG_PROF_COEF, l0);
    if (l0 < last) {
      CK(launch_inject_levels(s->lset, s->lv[l0].L, l0, last, s->stream));
      CK(launch_coef_levels(s->lset, s->lv[l0 + 1].L, l0 + 1, last, s->tr, s->stream));
    }
    CK(launch_factor_levels(s->lset, s->lv[l0].L, l0, last, mixed(s), dt, s->prm.n0, s->stream));
  }
  LevelBuf &c = s->lv[s->nlev - 1];
  ProfScope ps(s, MG_PROF_COARSE_FACTOR, l0);
  CK(launch_coarse_factor(c.L, dt, s->M, s->Minv, s->rs, s->cs, s->flag, s->stream));
  return MG_OK;
}

template <typename T> const LevelT<T> &view(const LevelBuf &b);
template <> const LevelT<double> &view<double>(const LevelBuf &b) { return b.L; }
template <> const LevelT<float> &view<float>(const LevelBuf &b) { return b.M; }
template <typename T> double nscale_of(const mg_state *s);
template <> double nscale_of<double>(const mg_state *) { return 1.0; }
template <> double nscale_of<float>(const mg_state *s) { return s->prm.n0; }

template <typename T> void shape_of(const LevelBuf &b, int &bx, int &by);
template <> void shape_of<double>(const LevelBuf &b, int &bx, int &by) { bx = b.sbx; by = b.sby; }
template <> void shape_of<float>(const LevelBuf &b, int &bx, int &by) { bx = b.sbx32; by = b.sby32; }

template <typename T>
int smooth(mg_state *s, int l, int color, cudaStream_t st) {
  ProfScope ps(s, MG_PROF_SMOOTH, l);
  int bx, by;
  shape_of<T>(s->lv[l], bx, by);
  CK(launch_smooth<T>(view<T>(s->lv[l]), color, st, bx, by));
  return MG_OK;
}

template <typename T> int level_fused(const LevelBuf &b);
template <> int level_fused<double>(const LevelBuf &b) { return b.fuse; }
template <> int level_fused<float>(const LevelBuf &b) { return b.fuse32; }

template <typename T> int sweep_shape(const LevelBuf &b);
template <> int sweep_shape<double>(const LevelBuf &b) { return b.sw; }
template <> int sweep_shape<float>(const LevelBuf &b) { return b.sw32; }

// nu red-black sweeps on level l: fused sweeps alternate between du and du2 (the last one
// lands in du; odd counts end with a copy), or pairs of half-sweep launches.
template <typename T>
int smooth_sweeps(mg_state *s, int l, int nu, cudaStream_t st) {
  if (s->prm.line_smoother) {
    // a sweep: z-line half sweeps (even columns, then odd), r-line half sweeps (even rows, then
    // odd), or both in that order (alternating lines)
    T *scr = reinterpret_cast<T *>(s->line_scr);
    const int lm = s->prm.line_smoother;
    for (int k = 0; k < nu; ++k) {
      if (lm & 1)
        for (int col = 0; col < 2; ++col) {
          ProfScope ps(s, MG_PROF_SMOOTH, l);
          CK(launch_zline<T>(view<T>(s->lv[l]), col, scr, st));
        }
      if (lm & 2)
        for (int row = 0; row < 2; ++row) {
          ProfScope ps(s, MG_PROF_SMOOTH, l);
          CK(launch_rline<T>(view<T>(s->lv[l]), row, st));
        }
    }
    return MG_OK;
  }
  const LevelT<T> &b = view<T>(s->lv[l]);
  int rc;
  if (!s->prm.fused_sweep || !level_fused<T>(s->lv[l])) {
    for (int k = 0; k < nu; ++k)
      for (int col = 0; col < 2; ++col)
        if ((rc = smooth<T>(s, l, col, st))) return rc;
    return MG_OK;
  }
  SweepIO<T> io;
  for (int k = 0; k < nu; ++k) {
    const bool fwd = (k % 2 == 0);
    for (int q = 0; q < 3; ++q) {
      io.in[q] = fwd ? b.du[q] : b.du2[q];
      io.out[q] = fwd ? b.du2[q] : b.du[q];
    }
    ProfScope ps(s, MG_PROF_SMOOTH, l);
    CK(launch_sweep<T>(b, io, sweep_shape<T>(s->lv[l]), st));
  }
  if (nu % 2)
    for (int q = 0; q < 3; ++q)
      CK(cudaMemcpyAsync(b.du[q], b.du2[q], s->lv[l].nodes * sizeof(T), cudaMemcpyDeviceToDevice, st));
  return MG_OK;
}

template <typename T> const CoarseSet<T> *coarse_set(const mg_state *s);
template <> const CoarseSet<double> *coarse_set<double>(const mg_state *s) { return s->cset64; }
template <> const CoarseSet<float> *coarse_set<float>(const mg_state *s) { return s->cset32; }
template <typename T> size_t coarse_smem(const mg_state *s);
template <> size_t coarse_smem<double>(const mg_state *s) { return s->cc_smem64; }
template <> size_t coarse_smem<float>(const mg_state *s) { return s->cc_smem32; }

// pre- (which = 1) or post-smoothing (2) sweeps on level l
int nu_of(const mg_state *s, int l, int which) {
  const int set = which == 1 ? s->lv[l].nu1 : s->lv[l].nu2;
  if (set >= 0) return set;
  const int side = std::max(s->lv[l].nr, s->lv[l].nz);
  if (s->prm.nu_tiny_n > 0 && side <= s->prm.nu_tiny_n) return which == 1 ? s->prm.nu_tiny1 : s->prm.nu_tiny2;
  const bool small = s->prm.nu_coarse_n > 0 && side <= s->prm.nu_coarse_n;
  if (which == 1) return small ? s->prm.nu_coarse1 : s->prm.nu1;
  return small ? s->prm.nu_coarse2 : s->prm.nu2;
}

template <typename T>
int vcycle(mg_state *s, int l, cudaStream_t st) {
  const LevelT<T> &b = view<T>(s->lv[l]);
  if (l == s->cc_from && l < s->nlev - 1) {
    ProfScope ps(s, MG_PROF_COARSE, l);
    CK(launch_coarse_cycle<T>(coarse_set<T>(s), s->prm.coarse_kernel_ctas, s->prm.coarse_kernel_threads,
                              coarse_smem<T>(s), (s->prm.pdl & PDL_COARSE) != 0, st));
    return MG_OK;
  }
  if (l == s->nlev - 1) {
    CK(launch_coarse_solve<T>(b, s->Minv, s->rs, s->cs, nscale_of<T>(s), st));
    return MG_OK;
  }
  const LevelT<T> &c = view<T>(s->lv[l + 1]);
  int rc;
  if ((rc = smooth_sweeps<T>(s, l, nu_of(s, l, 1), st))) return rc;
  {
    ProfScope ps(s, MG_PROF_RESTRICT, l);
    CK(launch_linres_restrict<T>(b, c, st));
  }
  if ((rc = vcycle<T>(s, l + 1, st))) return rc;
  {
    ProfScope ps(s, MG_PROF_PROLONG, l);
    CK(launch_prolong_add<T>(c, b, st));
  }
  return smooth_sweeps<T>(s, l, nu_of(s, l, 2), st);
}

// Per-field sums of squares of the linear residual f - J du on level l0 into dout[0..2]; in the
// mixed form this is the FP64 outer defect, also written as the next FP32 right-hand side.
int launch_norm(mg_state *s, int l0, cudaStream_t st) {
  LevelBuf &b = s->lv[l0];
  ProfScope ps(s, MG_PROF_LINRES, l0);
  if (mixed(s)) {
    CK(launch_outer_residual(b.L, b.M, s->prm.n0, s->partials, s->counter, s->dout, st));
  } else {
    CK(launch_linres<double>(b.L, b.L.du, b.L.f, b.L.r, s->partials, s->counter, s->dout, st));
  }
  return MG_OK;
}

// One iteration of the linear-solve loop: a V-cycle (in the mixed form: an FP32 cycle on the
// FP64 defect followed by x += e in FP64) and the residual norms.
int cycle_and_norm(mg_state *s, int l0, cudaStream_t st) {
  int rc;
  if (mixed(s)) {
    CK(launch_zero_du<float>(s->lv[l0].M, st));
    if ((rc = vcycle<float>(s, l0, st))) return rc;
    CK(launch_mixed_update(s->lv[l0].L, s->lv[l0].M, s->prm.n0, st));
  } else {
    if ((rc = vcycle<double>(s, l0, st))) return rc;
  }
  return launch_norm(s, l0, st);
}

double weighted(const mg_state *s, const double w[3]) {
  double m = 0.0;
  for (int q = 0; q < 3; ++q) {
    const double v = std::sqrt(s->hout[q]) / w[q];
    if (!(v == v)) return NAN;
    m = std::max(m, v);
  }
  return m;
}

// Host-driven loop (used while kernels are being timed, and when graphs are switched off).
int linear_solve_eager(mg_state *s, int l0, double eta, int max_cycles, const double w[3], double *hist, int *ncyc,
                       bool *ok) {
  CK(launch_zero_du<double>(s->lv[l0].L, s->stream));
  int rc = launch_norm(s, l0, s->stream);
  if (rc || (rc = sync_read(s, 3))) return rc;
  const double r0 = weighted(s, w);
  *ncyc = 0;
  *ok = true;
  if (hist) hist[0] = r0 > 0.0 ? 1.0 : 0.0;
  if (r0 == 0.0) return MG_OK;
  double rel = 1.0;
  while (rel > eta && *ncyc < max_cycles) {
    if ((rc = cycle_and_norm(s, l0, s->stream)) || (rc = sync_read(s, 3))) return rc;
    ++*ncyc;
    rel = weighted(s, w) / r0;
    if (hist) hist[*ncyc] = rel;
    if (!(rel == rel) || std::isinf(rel)) { *ok = false; return MG_OK; }
  }
  *ok = rel <= eta;
  return MG_OK;
}

// Record the device-side solve for root level l0 as a CUDA graph:
//   zero du -> norms -> init -> WHILE(cond) { V-cycle -> norms -> check }
// captured on a private stream and replayed on the state's stream.
int build_solve_graph(mg_state *s, int l0) {
  cudaStream_t cs = s->cap_stream;
  cudaGraph_t graph = nullptr;
  CK(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle h;
  int rc = MG_OK;
  const char *where = "";
  cudaGraphNodeParams cp = {};
  cudaGraph_t body = nullptr;
  cudaStreamCaptureStatus status;
  const cudaGraphNode_t *deps = nullptr;
  const cudaGraphEdgeData *edges = nullptr;
  size_t nd = 0;
  cudaGraphNode_t cnode;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 0, 0);
  if (e != cudaSuccess) { rc = MG_ECUDA; where = "conditional handle"; goto done; }
  set_capturing(true);
  e = cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { rc = MG_ECUDA; where = "begin capture"; goto done; }
  if (launch_zero_du<double>(s->lv[l0].L, cs) != cudaSuccess || launch_norm(s, l0, cs) != MG_OK ||
      launch_solve_init(s->ctl, s->dout, h, cs) != cudaSuccess) {
    rc = MG_ECUDA; where = "prefix launches";
  }
  s->vprefix[l0] = captured_launches();
  if (rc == MG_OK && (e = cudaStreamGetCaptureInfo(cs, &status, nullptr, nullptr, &deps, &edges, &nd)) != cudaSuccess) {
    rc = MG_ECUDA; where = "capture info";
  }
  if (rc == MG_OK) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if ((e = cudaGraphAddNode(&cnode, graph, deps, edges, nd, &cp)) != cudaSuccess) {
      rc = MG_ECUDA; where = "conditional node";
    } else if ((e = cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
               cudaSuccess) {
      rc = MG_ECUDA; where = "capture dependencies";
    }
  }
  {
    cudaGraph_t g2 = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g2);
    if (rc == MG_OK && e2 != cudaSuccess) { rc = MG_ECUDA; where = "end capture"; e = e2; }
  }
  if (rc != MG_OK) goto done;
  body = cp.conditional.phGraph_out[0];
  set_capturing(true);
  e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { rc = MG_ECUDA; where = "begin body capture"; goto done; }
  if (cycle_and_norm(s, l0, cs) != MG_OK || launch_solve_check(s->ctl, s->dout, h, cs) != cudaSuccess) {
    rc = MG_ECUDA; where = "body launches";
  }
  s->vbody[l0] = captured_launches();
  {
    cudaGraph_t g3 = nullptr;
    const cudaError_t e3 = cudaStreamEndCapture(cs, &g3);
    if (rc == MG_OK && e3 != cudaSuccess) { rc = MG_ECUDA; where = "end body capture"; e = e3; }
  }
  if (rc == MG_OK && (e = cudaGraphInstantiate(&s->vexec[l0], graph, 0)) != cudaSuccess) {
    rc = MG_ECUDA; where = "instantiate";
  }
done:
  set_capturing(false);
  cudaGetLastError();
  if (graph) cudaGraphDestroy(graph);
  if (rc != MG_OK) {
    s->vexec[l0] = nullptr;
    return fail(s, MG_ECUDA, "linear-solve graph: %s: %s", where, cudaGetErrorString(e));
  }
  return MG_OK;
}

// Device-side solve: the control block goes in, the graph runs, the control block comes back
// into the pinned host mirror, all on the state's stream without waiting.  The caller
// synchronises the stream and then calls linear_solve_graph_end.
int linear_solve_graph_begin(mg_state *s, int l0, double eta, int max_cycles, const double w[3]) {
  if (!s->vexec[l0]) {
    int rc = build_solve_graph(s, l0);
    if (rc) return rc;
  }
  SolveCtl *h = s->hctl;
  for (int q = 0; q < 3; ++q) h->w[q] = w[q];
  h->eta = eta;
  h->max_cycles = std::min(max_cycles, kMaxHist - 1);
  h->ncyc = 0;
  h->r0 = 0.0;
  h->rel = 0.0;
  CK(cudaMemcpyAsync(s->ctl, h, offsetof(SolveCtl, hist), cudaMemcpyHostToDevice, s->stream));
  CK(cudaGraphLaunch(s->vexec[l0], s->stream));
  CK(cudaMemcpyAsync(h, s->ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, s->stream));
  return MG_OK;
}

void linear_solve_graph_end(mg_state *s, int l0, double eta, double *hist, int *ncyc, bool *ok) {
  const SolveCtl *h = s->hctl;
  *ncyc = h->ncyc;
  count_launch(s->vprefix[l0] + h->ncyc * s->vbody[l0]);
  if (hist)
    for (int k = 0; k <= h->ncyc; ++k) hist[k] = h->hist[k];
  *ok = (h->r0 == 0.0) || (h->rel <= eta);
}

int linear_solve_graph(mg_state *s, int l0, double eta, int max_cycles, const double w[3], double *hist, int *ncyc,
                       bool *ok) {
  int rc = linear_solve_graph_begin(s, l0, eta, max_cycles, w);
  if (rc) return rc;
  CK(cudaStreamSynchronize(s->stream));
  linear_solve_graph_end(s, l0, eta, hist, ncyc, ok);
  return MG_OK;
}

bool use_graph(const mg_state *s, int max_cycles) {
  return s->prm.use_graphs && s->prof_kernel == 0 && max_cycles < kMaxHist;
}

void solve_weights(const double tn[3], double w[3]) {
  for (int q = 0; q < 3; ++q) w[q] = tn[q] > 0.0 ? tn[q] : 1.0;
}

// V-cycles on level l0 from du = 0 until the weighted residual drops by eta (tn: the per-field
// norms of the Newton residual's absolute terms, the weights of the test).
int linear_solve(mg_state *s, int l0, double eta, int max_cycles, const double tn[3], double *hist, int *ncyc,
                 bool *ok) {
  double w[3];
  solve_weights(tn, w);
  const int rc = use_graph(s, max_cycles) ? linear_solve_graph(s, l0, eta, max_cycles, w, hist, ncyc, ok)
                                          : linear_solve_eager(s, l0, eta, max_cycles, w, hist, ncyc, ok);
  if (rc == MG_OK) s->stats.vcycles += *ncyc;
  return rc;
}

void copy_state_async(mg_state *s, int l0, bool to_old) {
  LevelBuf &b = s->lv[l0];
  for (int q = 0; q < 3; ++q) {
    if (to_old) cudaMemcpyAsync(b.sv.uold[q], b.sv.u[q], b.nodes * sizeof(double), cudaMemcpyDeviceToDevice, s->stream);
    else cudaMemcpyAsync(b.sv.u[q], b.sv.uold[q], b.nodes * sizeof(double), cudaMemcpyDeviceToDevice, s->stream);
  }
}

// ---------------------------------------------------------------- batched form (persistent launch)
// Work items of a phase whose kernel runs nblocks thread blocks, per_round of them per round of a
// persistent CTA, `grain` rounds per item.
BPhase batch_phase(int kind, int level, int arg, int nblocks, int per_round, int grain) {
  BPhase p;
  p.kind = kind;
  p.level = level;
  p.arg = arg;
  p.nblocks = nblocks;
  p.grain = grain;
  const int rounds = (nblocks + per_round - 1) / per_round;
  p.ntiles = (rounds + grain - 1) / grain;
  return p;
}

// Whether a state's steady solve can run in the batched launch: the point smoother, the Picard
// Jacobian, the coarse-cycle kernel at or below every root level of the continuation, a
// coarsest level of at most 48 unknowns (shared-memory inverse), and a continuation that
// mg_solve_steady accepts.
bool batchable(const mg_state *s) {
  const LevelBuf &c = s->lv[s->nlev - 1];
  return s->nlev >= 2 && s->nlev <= kMaxLevelSet && s->prm.chain_from >= 1 && s->prm.chain_from < s->nlev &&
         !s->prm.line_smoother && !s->prm.full_jacobian && s->cc_from > 0 &&
         s->cc_from < s->nlev - 1 && s->prm.chain_from <= s->cc_from && 3 * c.L.ni * (c.nz - 1) <= 48 &&
         s->prof_kernel == 0;
}

// The program of a steady solve: program counter 0 ends the solve; then, for every level l the
// continuation marches on (0 .. chain_from), subprograms that each end in BK_RET, in the order
// of the host driver's launches:
//   E_INJECT      state and sources injected from level l - 1 (l >= 1)
//   E_START_COEF  coefficients and the steady residual sums of the current state (start data)
//   E_START       the same without the coefficients
//   E_BEGIN_USE   u -> u_old and the stored steady -F -> f (a step starting from start data)
//   E_BEGIN_COEF  u -> u_old, coefficients and the step's residual (f and the sums)
//   E_BEGIN       the same without the coefficients
//   E_NEWTON      one Newton iteration: injection and coefficients of the coarser levels, the
//                 factors of every level, the coarsest inverse, du = 0 and the initial norm;
//                 the V-cycle loop from E_NLOOP (pre-smoothing half sweeps and the
//                 residual-restriction per level down to the coarse-cycle kernel's first level,
//                 the coarse cycle, prolongation and post-smoothing back up; in the mixed form
//                 the FP32 cycle between zeroing its correction and the FP64 update), closed by
//                 the norm and its stopping test; from E_NUPD the update, the coefficients and
//                 the residual of the new state
//   E_RESTORE     u_old -> u (a rejected step)
//   E_PROLONG     the state prolonged from level l + 1 and the boundary values set (l < chain_from)
// The device coarse set of the levels c .. last (as setup_coarse_kernel builds the one of the
// coarse-cycle kernel, from level c instead of cc_from).
int batch_coarse_set(mg_state *s, int c) {
  if (s->bcs64[c]) return MG_OK;
  if (s->nlev - c > kMaxCoarseSet) return fail(s, MG_EINVAL, "batched coarse phase: %d levels", s->nlev - c);
  CoarseSet<double> h64 = {};
  CoarseSet<float> h32 = {};
  h64.n = h32.n = s->nlev - c;
  for (int q = 0; q < h64.n; ++q) {
    h64.nu1[q] = h32.nu1[q] = nu_of(s, c + q, 1);
    h64.nu2[q] = h32.nu2[q] = nu_of(s, c + q, 2);
    h64.lv[q] = s->lv[c + q].L;
    h32.lv[q] = s->lv[c + q].M;
  }
  h64.Minv = h32.Minv = s->Minv;
  h64.rs = h32.rs = s->rs;
  h64.cs = h32.cs = s->cs;
  h64.nscale = 1.0;
  h32.nscale = s->prm.n0;
  void *d64 = nullptr, *d32 = nullptr;
  CK(cudaMalloc(&d64, sizeof(h64)));
  if (cudaMalloc(&d32, sizeof(h32)) != cudaSuccess) {
    cudaFree(d64);
    return fail(s, MG_ECUDA, "batched coarse set");
  }
  s->bcs64[c] = static_cast<CoarseSet<double> *>(d64);
  s->bcs32[c] = static_cast<CoarseSet<float> *>(d32);
  CK(cudaMemcpy(d64, &h64, sizeof(h64), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d32, &h32, sizeof(h32), cudaMemcpyHostToDevice));
  return MG_OK;
}

int build_batch_program(mg_state *s) {
  if (s->bprog) return MG_OK;
  const int last = s->nlev - 1, g = s->bgrain, from = s->prm.chain_from;
  // the V-cycle of root level l0 descends level by level until the coarse phase's first level:
  // the first level with at most bcoarse_n intervals per side (never below the coarse-cycle
  // kernel's), or l0 itself
  int bcc = s->cc_from;
  for (int l = 1; l < s->cc_from; ++l)
    if (std::max(s->lv[l].nr, s->lv[l].nz) <= s->bcoarse_n) { bcc = l; break; }
  const bool m = mixed(s);
  auto cdiv = [](long a, long b) { return (int)((a + b - 1) / b); };
  auto grid328 = [&](const Level &L, int rows) { return cdiv(L.nr + 1, 32) * cdiv(rows, 8); };
  std::vector<BPhase> p;
  BPhase end = {};
  end.kind = BK_DONE;
  p.push_back(end);
  BPhase ret = {};
  ret.kind = BK_RET;
  std::memset(s->bent, 0, sizeof(s->bent));
  for (int l0 = 0; l0 <= from; ++l0) {
    const Level &L0 = s->lv[l0].L;
    int *E = s->bent[l0];
    const int nb_resid = cdiv(L0.nr + 1, 32) * cdiv(L0.nz - 1, 2);
    const int nb_copy = cdiv((long)(L0.nz + 1) * L0.P, kBatchThreads);
    if (l0 >= 1) {
      E[E_INJECT] = (int)p.size();
      p.push_back(batch_phase(BK_INJECT1, l0, 0, grid328(L0, L0.nz + 1), 1, g));
      p.push_back(ret);
    }
    E[E_START_COEF] = (int)p.size();
    p.push_back(batch_phase(BK_COEF0, l0, l0, grid328(L0, L0.nz + 1), 1, g));
    E[E_START] = (int)p.size();
    p.push_back(batch_phase(BK_RESID, l0, RESID_STEADY, nb_resid, 4, g));
    p.push_back(ret);
    E[E_BEGIN_USE] = (int)p.size();
    p.push_back(batch_phase(BK_COPY, l0, COPY_TO_OLD, nb_copy, 1, g));
    p.push_back(batch_phase(BK_COPY, l0, COPY_FSS_TO_F, nb_copy, 1, g));
    p.push_back(ret);
    E[E_BEGIN_COEF] = (int)p.size();
    p.push_back(batch_phase(BK_COPY, l0, COPY_TO_OLD, nb_copy, 1, g));
    p.push_back(batch_phase(BK_COEF0, l0, l0, grid328(L0, L0.nz + 1), 1, g));
    p.push_back(batch_phase(BK_RESID, l0, RESID_WRITE_F | RESID_DT, nb_resid, 4, g));
    p.push_back(ret);
    E[E_BEGIN] = (int)p.size();
    p.push_back(batch_phase(BK_COPY, l0, COPY_TO_OLD, nb_copy, 1, g));
    p.push_back(batch_phase(BK_RESID, l0, RESID_WRITE_F | RESID_DT, nb_resid, 4, g));
    p.push_back(ret);
    // one Newton iteration
    E[E_NEWTON] = (int)p.size();
    if (l0 < last) {
      const Level &C1 = s->lv[l0 + 1].L;
      p.push_back(batch_phase(BK_INJECT, l0 + 1, last, grid328(C1, C1.nz + 1) * (last - l0), 1, g));
      p.push_back(batch_phase(BK_COEFL, l0 + 1, last, grid328(C1, C1.nz + 1) * (last - l0), 1, g));
    }
    p.push_back(batch_phase(BK_FACTORL, l0, last, grid328(L0, L0.nz + 1) * (last - l0 + 1), 1, g));
    p.push_back(batch_phase(BK_CFACT, last, 0, 1, 1, 1));
    p.push_back(batch_phase(BK_ZERO64, l0, 0, nb_copy, 1, g));
    const int nb_norm = m ? grid328(L0, L0.nz - 1) : cdiv(L0.nr + 1, 32) * cdiv(L0.nz - 1, 2);
    p.push_back(batch_phase(BK_NORM0, l0, 0, nb_norm, m ? 1 : 4, g));
    E[E_NLOOP] = (int)p.size();
    if (m) p.push_back(batch_phase(BK_ZERO32, l0, 0, nb_copy, 1, g));
    auto halves = [&](int l, int nu) {
      const Level &L = s->lv[l].L;
      const int nb = cdiv((long)(L.nz / 2) * L.ni, kBatchThreads);
      for (int k = 0; k < nu; ++k)
        for (int col = 0; col < 2; ++col) p.push_back(batch_phase(m ? BK_HALF32 : BK_HALF64, l, col, nb, 1, g));
    };
    const int c0 = std::max(l0, bcc);
    int rc = batch_coarse_set(s, c0);
    if (rc) return rc;
    for (int l = l0; l < c0; ++l) {
      halves(l, nu_of(s, l, 1));
      const Level &C = s->lv[l + 1].L;
      p.push_back(batch_phase(m ? BK_RESTR32 : BK_RESTR64, l, 0, cdiv(C.nr + 1, 16) * cdiv(C.nz - 1, 3), 1, g));
    }
    p.push_back(batch_phase(m ? BK_COARSE32 : BK_COARSE64, c0, 0, 1, 1, 1));
    for (int l = c0 - 1; l >= l0; --l) {
      const Level &F = s->lv[l].L;
      p.push_back(batch_phase(m ? BK_PROL32 : BK_PROL64, l, 0, cdiv((long)F.ni * (F.nz - 1), kBatchThreads), 1, g));
      halves(l, nu_of(s, l, 2));
    }
    if (m) p.push_back(batch_phase(BK_MIXUPD, l0, 0, cdiv((long)L0.ni * (L0.nz - 1), kBatchThreads), 1, g));
    p.push_back(batch_phase(BK_NORMC, l0, 0, nb_norm, m ? 1 : 4, g));
    E[E_NUPD] = (int)p.size();
    p.push_back(batch_phase(BK_UPDATE, l0, 0, grid328(L0, L0.nz - 1), 1, g));
    p.push_back(batch_phase(BK_COEF0, l0, l0, grid328(L0, L0.nz + 1), 1, g));
    p.push_back(batch_phase(BK_RESID, l0, RESID_WRITE_F | RESID_STEADY | RESID_DT, nb_resid, 4, g));
    p.push_back(ret);
    E[E_RESTORE] = (int)p.size();
    p.push_back(batch_phase(BK_COPY, l0, COPY_FROM_OLD, nb_copy, 1, g));
    p.push_back(ret);
    if (l0 < from) {
      E[E_PROLONG] = (int)p.size();
      p.push_back(batch_phase(BK_PROLST, l0, 0, cdiv((long)(L0.nr + 1) * (L0.nz + 1), kBatchThreads), 1, g));
      p.push_back(batch_phase(BK_DIRI, l0, 0, 1, 1, 1));
      p.push_back(ret);
    }
  }
  if ((int)p.size() > kBatchMaxProg) return fail(s, MG_EINVAL, "batched program too long (%d phases)", (int)p.size());
  for (const BPhase &q : p)
    if (q.ntiles >= (1 << 20)) return fail(s, MG_EINVAL, "batched program: a phase of %d work items", q.ntiles);
  s->host_prog_ntiles0 = p[s->bent[1][E_INJECT]].ntiles;
  void *d = nullptr;
  CK(cudaMalloc(&d, p.size() * sizeof(BPhase)));
  if (cudaMemcpy(d, p.data(), p.size() * sizeof(BPhase), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    return fail(s, MG_ECUDA, "batched program upload");
  }
  s->bprog = static_cast<BPhase *>(d);
  return MG_OK;
}

// The descriptor of state s's steady solve to tol: parameters and the start of the solve
// (the injection onto level 1 runs first).
void batch_describe(mg_state *s, double tol, BatchInst &I) {
  std::memset(&I, 0, sizeof(I));
  I.prog = s->bprog;
  std::memcpy(I.ent, s->bent, sizeof(I.ent));
  I.last = s->nlev - 1;
  I.mixed = mixed(s) ? 1 : 0;
  I.max_cycles = std::min(s->prm.max_vcycles, kMaxHist - 1);
  I.S = s->lset;
  for (int l = 0; l < kMaxLevelSet && l < kMaxLevels; ++l) {
    I.cs64[l] = s->bcs64[l];
    I.cs32[l] = s->bcs32[l];
  }
  I.tr = s->tr;
  I.n0 = s->prm.n0;
  I.ctl = s->ctl;
  I.partials = s->partials;
  I.dout = s->dout;
  I.Minv = s->Minv;
  I.rs = s->rs;
  I.cs = s->cs;
  I.flag = s->flag;
  for (int q = 0; q < 3; ++q) I.fss[q] = s->fss[q];
  BatchMarch &M = I.m;
  M.tol = tol;
  M.dt1 = s->prm.dt1;
  M.dt_max = s->prm.dt_max;
  M.dt_growth = s->prm.dt_growth;
  M.ntol = s->prm.newton_tol > 0.0 ? s->prm.newton_tol : 0.1 * tol;
  M.rel = s->prm.newton_tol_rel;
  M.limit = s->prm.corr_limit_frac * std::fabs(s->prm.V_anode - s->prm.V_cathode);
  M.eta_p = s->prm.eta;
  M.Vc = s->prm.V_cathode;
  M.Va = s->prm.V_anode;
  M.from = s->prm.chain_from;
  M.max_steps = s->prm.max_steps;
  M.max_newton = s->prm.max_newton;
  M.eta_adapt = s->prm.eta_adapt;
  M.stage = 0;  // the injection onto level 1 runs first
  M.lvl = 1;
  M.start_valid = 0;
  M.steady_rho = s->stats.steady_rho;
  M.dt_last = s->stats.dt_last;
  for (int q = 0; q < 3; ++q) M.srho[q] = s->stats.rho[q];
  I.claim = 0ull;
  // ring entry of phase 0: (sequence 0 << 32) | (program counter << 20) | work items
  const int pc0 = s->bent[1][E_INJECT];
  I.ring[0] = ((unsigned long long)(unsigned)pc0 << 20) | (unsigned)s->host_prog_ntiles0;
  I.ring[1] = I.ring[2] = I.ring[3] = ~0ull;
  I.done = 0u;
}

// The statistics and start data of a finished batched solve into the state.
void batch_collect(mg_state *s, const BatchInst &I) {
  const BatchMarch &M = I.m;
  mg_stats &t = s->stats;
  t.steps_accepted += M.steps_accepted;
  t.steps_rejected += M.steps_rejected;
  t.newton_iterations += M.newton_iterations;
  t.vcycles += M.vcycles;
  t.coarse_steps += M.coarse_steps;
  t.coarse_newton += M.coarse_newton;
  t.coarse_vcycles += M.coarse_vcycles;
  if (M.steps_accepted + M.steps_rejected > 0) t.last_newton = M.last_newton;
  for (int q = 0; q < 3; ++q) t.rho[q] = M.srho[q];
  t.steady_rho = M.steady_rho;
  t.dt_last = M.dt_last;
  t.sim_time += M.sim_time;
  for (int q = 0; q < 16; ++q) s->start_sums[q] = M.start_sums[q];
  s->start_valid = M.start_valid != 0;
}

// One backward-Euler step on level l0 (eq. 7 by Newton-Raphson on eq. 14).
// Returns MG_OK (accepted), MG_ENOCONV or MG_ENONFINITE (rejected; state restored).
// coef_current: the face coefficients of level l0 are those of the current state (the caller
// evaluated a residual at this state and changed nothing since).
// A Newton iteration enqueues the hierarchy set-up, the device-side linear solve, the update
// and the next residual, then waits once and reads the solve's control block, the update's
// checks and the new residual norms together.
// Full-Jacobian Newton step on level l0 (mu, D functions of |E|): the multigrid solve of the
// Picard system has left du; while the full defect  max_f ||f - J_full du||_f / w_f  exceeds
// eta * f0 (f0 = the same for f, the Newton residual's weighted norm), solve the Picard system
// for the defect and add the correction.  du ends as the accumulated step.
int full_jacobian_correct(mg_state *s, int l0, double eta, const double tn[3], double f0, int *ncyc, bool *ok) {
  LevelBuf &b = s->lv[l0];
  cudaStream_t st = s->stream;
  const size_t bytes = b.nodes * sizeof(double);
  double w[3];
  solve_weights(tn, w);
  for (int q = 0; q < 3; ++q) {
    CK(cudaMemcpyAsync(s->fj_f[q], b.L.f[q], bytes, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(s->fj_d[q], b.L.du[q], bytes, cudaMemcpyDeviceToDevice, st));
  }
  *ok = false;
  *ncyc = 0;
  for (int c = 0; c <= s->prm.max_corrections; ++c) {
    CK(launch_full_defect(b.L, b.sv, s->tr, s->fj_f, s->fj_d, s->partials, s->counter, s->dout, st));
    int rc = sync_read(s, 3);
    if (rc) return rc;
    const double r = weighted(s, w);
    if (!(r == r)) break;
    if (r <= eta * f0) { *ok = true; break; }
    if (c == s->prm.max_corrections) break;
    // the Picard solve of J_P e = defect, relative to the defect
    int nc = 0;
    bool lok = false;
    rc = linear_solve(s, l0, eta, s->prm.max_vcycles, tn, nullptr, &nc, &lok);
    if (rc) return rc;
    *ncyc += nc;
    s->stats.vcycles -= nc;  // counted by the caller with the first solve's cycles
    if (!lok) break;
    CK(launch_add3(s->fj_d, b.L.du, b.nodes, st));
  }
  for (int q = 0; q < 3; ++q) CK(cudaMemcpyAsync(b.L.du[q], s->fj_d[q], bytes, cudaMemcpyDeviceToDevice, st));
  return MG_OK;
}

// steady_rho (may be NULL): on acceptance after at least one Newton iteration, the steady
// residual of the new state (from the same residual launch), else -1.
// use_start: the state's start data (start_data, or the last residual launch of the previous
// accepted step) stand in for the step's first residual launch (coefficients current too).
int step(mg_state *s, int l0, double dt, double tol, int *newton_out, bool coef_current = false,
         double *steady_rho = nullptr, bool use_start = false) {
  LevelBuf &b = s->lv[l0];
  copy_state_async(s, l0, true);
  CK(cudaGetLastError());
  const double limit = s->prm.corr_limit_frac * std::fabs(s->prm.V_anode - s->prm.V_cathode);
  int rc;
  int reason = MG_ENOCONV;
  double rho[3], tn[3];
  if (steady_rho) *steady_rho = -1.0;
  double rho_steady[3] = {-1.0, -1.0, -1.0};
  double cand[16];
  if (use_start && s->start_valid) {
    start_norms(s, dt, rho, tn);
    for (int q = 0; q < 3; ++q)
      CK(cudaMemcpyAsync(b.L.f[q], s->fss[q], b.nodes * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
  } else {
    rc = residual(s, l0, dt, true, nullptr, rho, tn, !coef_current);
    if (rc) return rc;
  }
  for (int it = 0; it <= s->prm.max_newton; ++it) {
    for (int q = 0; q < 3; ++q) s->stats.rho[q] = rho[q];
    const double rmax = std::max(rho[0], std::max(rho[1], rho[2]));
    if (!(rmax == rmax) || std::isinf(rmax)) { reason = MG_ENONFINITE; *newton_out = it; break; }
    if (rmax <= tol) {
      if (steady_rho && it > 0) *steady_rho = std::max(rho_steady[0], std::max(rho_steady[1], rho_steady[2]));
      if (it > 0) {  // the accepted state's start data come from its residual launch
        for (int q = 0; q < 16; ++q) s->start_sums[q] = cand[q];
        s->start_valid = true;
      }
      *newton_out = it;
      s->stats.newton_iterations += it;
      s->stats.last_newton = it;
      return MG_OK;
    }
    if (it == s->prm.max_newton) { *newton_out = it; break; }
    s->start_valid = false;  // this iteration's residual launch overwrites fss and the sums
    int ncyc;
    bool ok;
    // inexact-Newton forcing term: drive the linear residual only to half the Newton target
    const double eta = s->prm.eta_adapt ? std::max(s->prm.eta, std::min(0.1, 0.5 * tol / rmax)) : s->prm.eta;
    double w[3];
    solve_weights(tn, w);
    rc = build_hierarchy(s, l0, dt);
    if (rc) return rc;
    const bool graph = use_graph(s, s->prm.max_vcycles);
    const bool full = s->prm.full_jacobian != 0;
    if (graph) rc = linear_solve_graph_begin(s, l0, eta, s->prm.max_vcycles, w);
    else rc = linear_solve_eager(s, l0, eta, s->prm.max_vcycles, w, nullptr, &ncyc, &ok);
    if (rc) return rc;
    if (full) {
      // the defect corrections need the Picard step first
      if (graph) {
        CK(cudaStreamSynchronize(s->stream));
        linear_solve_graph_end(s, l0, eta, nullptr, &ncyc, &ok);
      }
      if (ok) {
        int nc2 = 0;
        if ((rc = full_jacobian_correct(s, l0, eta, tn, rmax, &nc2, &ok))) return rc;
        ncyc += nc2;
      }
    }
    // u += du (max |dV| and the non-finite flag into dout[16..17]), then the residual at the new
    // state (into dout[0..5], its steady rows' sums and start data into dout[6..15] and fss);
    // used only if the update is accepted
    CK(launch_update(b.L, b.sv, s->partials, s->counter, s->dout + 16, s->stream));
    if ((rc = residual_launch(s, l0, dt, true, nullptr, true, true))) return rc;
    rc = sync_read(s, 18);
    if (rc) return rc;
    if (graph && !full) linear_solve_graph_end(s, l0, eta, nullptr, &ncyc, &ok);
    s->stats.vcycles += ncyc;
    if (!ok) { *newton_out = it + 1; reason = MG_ENOCONV; break; }
    if (s->hout[17] != 0.0) { *newton_out = it + 1; reason = MG_ENONFINITE; break; }
    if (s->hout[16] > limit) { *newton_out = it + 1; reason = MG_ENOCONV; break; }
    residual_norms(s, rho, tn);
    for (int q = 0; q < 16; ++q) cand[q] = s->hout[q];
    for (int q = 0; q < 3; ++q) {
      const double fn = std::sqrt(s->hout[6 + q]), t = std::sqrt(s->hout[9 + q]);
      rho_steady[q] = fn == 0.0 ? 0.0 : (t > 0.0 ? fn / t : INFINITY);
    }
  }
  s->stats.newton_iterations += *newton_out;
  s->stats.last_newton = *newton_out;
  copy_state_async(s, l0, false);
  CK(cudaGetLastError());
  return reason;
}

// March on level l0 with the Delta-t ramp until the steady residual <= tol.  Each step is
// solved to the per-step tolerance (default 0.1 tol: a step's residual measure includes the
// time-derivative terms, the steady one does not) or, with newton_tol_rel > 0, to
// newton_tol_rel x the steady residual at the step's start when that is larger.
int march(mg_state *s, int l0, double dt_start, double tol) {
  double dt = dt_start, dt_prev = -1.0;
  const double ntol = s->prm.newton_tol > 0.0 ? s->prm.newton_tol : 0.1 * tol;
  const double rel = s->prm.newton_tol_rel;
  bool coef_current = false;  // face coefficients of level l0 at the current state
  double r_start = 0.0;       // steady residual of the current state
  auto steady_of_start = [&]() {  // the steady residual of the start state
    double m = 0.0;
    for (int q = 0; q < 3; ++q) {
      const double fn = std::sqrt(s->start_sums[6 + q]), t = std::sqrt(s->start_sums[9 + q]);
      m = std::max(m, fn == 0.0 ? 0.0 : (t > 0.0 ? fn / t : INFINITY));
    }
    return m;
  };
  // one residual launch gives the first step's residual and the steady residual of the start
  {
    const int rc = start_data(s, l0, true);
    if (rc) return rc;
    coef_current = true;
    r_start = steady_of_start();
  }
  for (int n = 0; n < s->prm.max_steps; ++n) {
    int newton = 0;
    const double step_tol = std::max(ntol, rel * r_start);
    double r_step = -1.0;
    int rc = step(s, l0, dt, step_tol, &newton, coef_current, &r_step, true);
    coef_current = false;
    if (rc == MG_ECUDA) return rc;
    s->stats.dt_last = dt;
    if (rc == MG_OK) {
      s->stats.steps_accepted++;
      s->stats.sim_time += dt;
      // the accepted step ended on a residual at this very state: its coefficients stand, and
      // they serve the next step's first residual too; that launch also summed the steady rows
      // (after at least one Newton iteration), otherwise evaluate them here
      double r = r_step;
      if (r < 0.0) {
        // accepted without a Newton iteration: the state is the start state
        if (!s->start_valid && (rc = start_data(s, l0, false))) return rc;
        r = steady_of_start();
      }
      coef_current = true;
      s->stats.steady_rho = r;
      r_start = r;
      if (r <= tol) return MG_OK;
      dt_prev = dt;
      dt = std::min(dt * s->prm.dt_growth, s->prm.dt_max);
    } else {
      s->stats.steps_rejected++;
      if (dt_prev > 0.0 && dt > dt_prev) {
        dt = dt_prev;
      } else {
        dt *= 0.5;
        if (dt_prev > 0.0) dt_prev = std::min(dt_prev, dt);
      }
    }
  }
  return fail(s, MG_EREJECT, "march: steady residual not reached in %d steps", s->prm.max_steps);
}

// Device copy of every level's views (pointers and geometry scalars are fixed after mg_create).
int upload_level_set(mg_state *s) {
  if (s->nlev > kMaxLevelSet) return fail(s, MG_EINVAL, "too many levels (%d)", s->nlev);
  LevelSet h;
  std::memset(&h, 0, sizeof(h));
  for (int l = 0; l < s->nlev; ++l) {
    h.L[l] = s->lv[l].L;
    h.M[l] = s->lv[l].M;
    h.sv[l] = s->lv[l].sv;
  }
  CK(cudaMemcpy(s->lset, &h, sizeof(h), cudaMemcpyHostToDevice));
  return MG_OK;
}

// Choose the first level handled by the persistent coarse-cycle kernel (all levels whose
// larger side has at most coarse_kernel_n intervals) and upload the level views it needs.
int setup_coarse_kernel(mg_state *s) {
  s->cc_from = -1;
  if (s->prm.coarse_kernel_n <= 0 || s->prm.line_smoother) return MG_OK;
  for (int l = 1; l < s->nlev - 1; ++l)
    if (std::max(s->lv[l].nr, s->lv[l].nz) <= s->prm.coarse_kernel_n) { s->cc_from = l; break; }
  if (s->cc_from < 0 || s->nlev - s->cc_from > kMaxCoarseSet) { s->cc_from = -1; return MG_OK; }
  CoarseSet<double> h64 = {};
  CoarseSet<float> h32 = {};
  h64.n = h32.n = s->nlev - s->cc_from;
  for (int q = 0; q < h64.n; ++q) {
    h64.nu1[q] = h32.nu1[q] = nu_of(s, s->cc_from + q, 1);
    h64.nu2[q] = h32.nu2[q] = nu_of(s, s->cc_from + q, 2);
  }
  h64.Minv = h32.Minv = s->Minv;
  h64.rs = h32.rs = s->rs;
  h64.cs = h32.cs = s->cs;
  h64.nscale = 1.0;
  h32.nscale = s->prm.n0;
  for (int q = 0; q < h64.n; ++q) {
    h64.lv[q] = s->lv[s->cc_from + q].L;
    h32.lv[q] = s->lv[s->cc_from + q].M;
  }
  CK(cudaMemcpy(s->cset64, &h64, sizeof(h64), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->cset32, &h32, sizeof(h32), cudaMemcpyHostToDevice));
  constexpr size_t kCoarseSmemLimit = 200 * 1024;
  s->cc_smem64 = prepare_coarse_smem(h64, kCoarseSmemLimit);
  s->cc_smem32 = mixed(s) ? prepare_coarse_smem(h32, kCoarseSmemLimit) : 0;
  return MG_OK;
}

int check_where(mg_state *s, int where) {
  if (where != MG_HOST && where != MG_DEVICE) return fail(s, MG_EINVAL, "where must be MG_HOST or MG_DEVICE");
  return MG_OK;
}

}  // namespace

// ---------------------------------------------------------------- autotuner
namespace {
// Mean device time of `reps` launches of the smoother with shape (bx, by) on level l.
template <typename T>
int time_shape(mg_state *s, int l, int bx, int by, int reps, cudaEvent_t e0, cudaEvent_t e1, float *ms) {
  const LevelT<T> &L = view<T>(s->lv[l]);
  for (int r = 0; r < 2; ++r) CK(launch_smooth<T>(L, r & 1, s->stream, bx, by));
  CK(cudaEventRecord(e0, s->stream));
  for (int r = 0; r < reps; ++r) CK(launch_smooth<T>(L, r & 1, s->stream, bx, by));
  CK(cudaEventRecord(e1, s->stream));
  CK(cudaEventSynchronize(e1));
  CK(cudaEventElapsedTime(ms, e0, e1));
  *ms /= reps;
  return MG_OK;
}

template <typename T>
int time_sweep(mg_state *s, int l, int shape, int reps, cudaEvent_t e0, cudaEvent_t e1, float *ms) {
  const LevelT<T> &L = view<T>(s->lv[l]);
  SweepIO<T> io;
  for (int q = 0; q < 3; ++q) { io.in[q] = L.du[q]; io.out[q] = L.du2[q]; }
  for (int r = 0; r < 2; ++r) CK(launch_sweep<T>(L, io, shape, s->stream));
  CK(cudaEventRecord(e0, s->stream));
  for (int r = 0; r < reps; ++r) CK(launch_sweep<T>(L, io, shape, s->stream));
  CK(cudaEventRecord(e1, s->stream));
  CK(cudaEventSynchronize(e1));
  CK(cudaEventElapsedTime(ms, e0, e1));
  *ms /= reps;
  return MG_OK;
}
}  // namespace

// ================================================================ C ABI
extern "C" {

void mg_params_default(mg_params *p) {
  std::memset(p, 0, sizeof(*p));
  p->V_cathode = -200.0; p->V_anode = 0.0;
  p->mu_e = 30.0; p->D_e = 60.0; p->mu_p = 0.15; p->D_p = 0.0038;
  p->table = nullptr; p->table_rows = 0;
  p->precision = MG_FP64;
  p->pressure_factor = 1.0;
  p->nu1 = 4; p->nu2 = 4; p->coarsest = 2;
  p->max_vcycles = 60; p->max_newton = 10; p->max_steps = 400;
  p->eta = 1e-3; p->newton_tol = 0.0; p->corr_limit_frac = 0.5;
  p->dt1 = 1e-9; p->dt_growth = 5.0; p->dt_max = 1e-6;
  p->n0 = 1e14;
  p->use_graphs = 1;
  p->fused_sweep = 1;
  p->guess_dt_max = 1e-3;
  p->guess_level = 0;
  p->guess_dt_start = 1e-8;
  p->eta_adapt = 1;
  p->nu_coarse_n = 64; p->nu_coarse1 = 2; p->nu_coarse2 = 2;
  p->nu_tiny_n = 8; p->nu_tiny1 = 1; p->nu_tiny2 = 1;
  p->chain_from = 1;
  p->pdl = PDL_SMOOTH | PDL_COARSE;
  p->wall_dirichlet = 0;
  p->newton_tol_rel = 0.1;
  p->full_jacobian = 0;
  p->max_corrections = 20;
  p->line_smoother = 0;
  p->coarse_kernel_n = 16;
  p->coarse_kernel_ctas = 1;
  p->coarse_kernel_threads = 512;
}

static int validate(const mg_grid *g, const mg_params *p, std::string *why) {
  if (!g || !p) { *why = "null grid or params"; return MG_EINVAL; }
  if (!pow2(g->nr) || !pow2(g->nz)) { *why = "nr and nz must be powers of two >= 2"; return MG_EINVAL; }
  if (!(g->R > 0.0) || !g->z) { *why = "R must be positive and z given"; return MG_EINVAL; }
  for (int j = 0; j < g->nz; ++j)
    if (!(g->z[j + 1] > g->z[j])) { *why = "z must increase strictly"; return MG_EINVAL; }
  if (p->coarsest < 2 || p->coarsest > 8) { *why = "coarsest must be in 2..8"; return MG_EINVAL; }
  if (p->nu1 < 0 || p->nu2 < 0 || p->nu1 + p->nu2 < 1) { *why = "need at least one smoothing sweep"; return MG_EINVAL; }
  if (p->nu_coarse_n < 0 || (p->nu_coarse_n > 0 && (p->nu_coarse1 < 0 || p->nu_coarse2 < 0 ||
                                                     p->nu_coarse1 + p->nu_coarse2 < 1))) {
    *why = "nu_coarse_n >= 0 and, when set, at least one coarse smoothing sweep";
    return MG_EINVAL;
  }
  if (p->wall_dirichlet != 0 && p->wall_dirichlet != 1) { *why = "wall_dirichlet must be 0 or 1"; return MG_EINVAL; }
  if (!(p->newton_tol_rel >= 0.0 && p->newton_tol_rel < 1.0)) { *why = "newton_tol_rel must be in [0, 1)"; return MG_EINVAL; }
  if (p->full_jacobian != 0 && p->full_jacobian != 1) { *why = "full_jacobian must be 0 or 1"; return MG_EINVAL; }
  if (p->max_corrections < 1 || p->max_corrections > 100) { *why = "max_corrections must be in 1..100"; return MG_EINVAL; }
  if (p->line_smoother < 0 || p->line_smoother > 3) { *why = "line_smoother must be 0, 1, 2 or 3"; return MG_EINVAL; }
  if ((p->line_smoother & 2) && (p->wall_dirichlet ? g->nr : g->nr + 1) > kRlineMax) {
    *why = "r-lines need rows of at most 512 unknowns";
    return MG_EINVAL;
  }
  if (p->pdl < 0 || p->pdl > PDL_ALL) { *why = "pdl: a combination of the PDL kernel-kind bits"; return MG_EINVAL; }
  if (p->nu_tiny_n < 0 || (p->nu_tiny_n > 0 && (p->nu_tiny1 < 0 || p->nu_tiny2 < 0 || p->nu_tiny1 + p->nu_tiny2 < 1))) {
    *why = "nu_tiny_n >= 0 and, when set, at least one smoothing sweep on those levels";
    return MG_EINVAL;
  }
  if (!(p->pressure_factor > 0.0) || !(p->D_e > 0.0) || !(p->D_p > 0.0) || p->mu_e < 0 || p->mu_p < 0) {
    *why = "transport coefficients must be positive"; return MG_EINVAL;
  }
  if (p->table) {
    if (p->table_rows < 2) { *why = "table needs >= 2 rows"; return MG_EINVAL; }
    for (int r = 0; r < p->table_rows; ++r) {
      if (r > 0 && !(p->table[5 * r] > p->table[5 * (r - 1)])) { *why = "table |E| must increase"; return MG_EINVAL; }
      if (!(p->table[5 * r + 2] > 0.0) || !(p->table[5 * r + 4] > 0.0)) { *why = "table D must be positive"; return MG_EINVAL; }
    }
  }
  if (p->precision != MG_FP64 && p->precision != MG_MIXED) { *why = "unknown precision"; return MG_EINVAL; }
  if (p->precision == MG_MIXED && !(p->n0 > 0.0)) { *why = "n0 must be positive"; return MG_EINVAL; }
  if (p->coarse_kernel_n > 0 && (p->coarse_kernel_ctas < 1 || p->coarse_kernel_ctas > 8 ||
                                 p->coarse_kernel_threads < 32 || p->coarse_kernel_threads > 1024 ||
                                 p->coarse_kernel_threads % 32)) {
    *why = "coarse kernel: 1..8 CTAs of 32..1024 threads (multiple of 32)";
    return MG_EINVAL;
  }
  int lnr[kMaxLevels], lnz[kMaxLevels];
  const int n = plan_levels(g->nr, g->nz, p->coarsest, lnr, lnz);
  if (3 * (lnr[n - 1] + 1) * (lnz[n - 1] - 1) > kMaxCoarse) { *why = "coarsest level too large (too anisotropic grid)"; return MG_EINVAL; }
  return MG_OK;
}

size_t mg_workspace_bytes(const mg_grid *g, const mg_params *p) {
  std::string why;
  if (validate(g, p, &why) != MG_OK) return 0;
  int lnr[kMaxLevels], lnz[kMaxLevels];
  const int n = plan_levels(g->nr, g->nz, p->coarsest, lnr, lnz);
  mg_state tmp;
  Carver c{nullptr, 0};
  carve(c, &tmp, n, lnr, lnz, p->table ? p->table_rows : 0, p->precision == MG_MIXED,
        p->line_smoother != 0);
  return c.off;
}

int mg_create(const mg_grid *g, const mg_params *p, void *stream, void *workspace, size_t workspace_bytes,
              mg_state **out) {
  if (!out) return MG_EINVAL;
  *out = nullptr;
  std::string why;
  int v = validate(g, p, &why);
  if (v != MG_OK) return v;
  mg_state *s = new (std::nothrow) mg_state();
  if (!s) return MG_ENOMEM;
  s->prm = *p;
  s->nr = g->nr; s->nz = g->nz; s->R = g->R;
  s->z.assign(g->z, g->z + g->nz + 1);
  if (p->table) {
    s->table_h.assign(p->table, p->table + 5 * p->table_rows);
    s->prm.table = s->table_h.data();
  }
  s->stream = (cudaStream_t)stream;
  int lnr[kMaxLevels], lnz[kMaxLevels];
  s->nlev = plan_levels(g->nr, g->nz, p->coarsest, lnr, lnz);
  Carver sizer{nullptr, 0};
  carve(sizer, s, s->nlev, lnr, lnz, p->table ? p->table_rows : 0, p->precision == MG_MIXED,
        p->line_smoother != 0);
  const size_t need = sizer.off;
  if (workspace) {
    if (workspace_bytes < need || ((uintptr_t)workspace & (kAlign - 1))) {
      delete s;
      return MG_ENOMEM;
    }
    s->ws = workspace; s->owns_ws = false;
  } else {
    if (cudaMalloc(&s->ws, need) != cudaSuccess) { delete s; return MG_ENOMEM; }
    s->owns_ws = true;
  }
  s->ws_bytes = need;
  if (cudaMallocHost(&s->hout, 24 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&s->hctl, sizeof(SolveCtl)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    if (s->owns_ws) cudaFree(s->ws);
    delete s;
    return MG_ECUDA;
  }
  Carver c{(char *)s->ws, 0};
  carve(c, s, s->nlev, lnr, lnz, p->table ? p->table_rows : 0, p->precision == MG_MIXED,
        p->line_smoother != 0);
  int rc = MG_OK;
  // zero everything once (electrode rows of du stay zero forever)
  if (cudaMemsetAsync(s->ws, 0, need, s->stream) != cudaSuccess) rc = fail(s, MG_ECUDA, "memset workspace");
  // geometry per level
  std::vector<double> geo;
  for (int l = 0; l < s->nlev && rc == MG_OK; ++l) {
    LevelBuf &b = s->lv[l];
    std::vector<double> zl;
    for (int j = 0; j <= g->nz; j += (1 << l)) zl.push_back(g->z[j]);
    const int glen = std::max(b.nr, b.nz) + 2;
    host_geometry(zl, b.nr, g->R, geo, glen);
    b.L.dr = g->R / b.nr;
    b.M.dr = (float)(g->R / b.nr);
    b.L.idr = 1.0 / b.L.dr;
    b.M.idr = (float)b.L.idr;
    b.L.ni = b.M.ni = p->wall_dirichlet ? b.nr : b.nr + 1;
    b.L.pdl = b.M.pdl = p->pdl;
    if (cudaMemcpyAsync(b.geo, geo.data(), geo.size() * sizeof(double), cudaMemcpyHostToDevice, s->stream) !=
        cudaSuccess)
      rc = fail(s, MG_ECUDA, "geometry copy");
    std::vector<float> geo32(geo.begin(), geo.end());
    if (b.geo32 && cudaMemcpyAsync(b.geo32, geo32.data(), geo32.size() * sizeof(float), cudaMemcpyHostToDevice,
                                   s->stream) != cudaSuccess)
      rc = fail(s, MG_ECUDA, "geometry copy (FP32)");
    // node arrays of the Poisson face conductances (r-face (i+1/2, j) and z-face (i, j+1/2), stored
    // at their lower node) and of (e/eps0) x control volume (x n0 for the FP32 copies)
    {
      const double *dz = geo.data(), *dzc = dz + glen, *volr = dz + 2 * glen;
      std::vector<double> nd(3 * b.nodes, 0.0);
      double *gR = nd.data(), *gZ = gR + b.nodes, *Ak = gZ + b.nodes;
      for (int j = 0; j <= b.nz; ++j)
        for (int i = 0; i <= b.nr; ++i) {
          const size_t k = (size_t)j * b.P + i;
          if (i < b.nr) gR[k] = (i + 0.5) * dzc[j];
          if (j < b.nz) gZ[k] = volr[i] / dz[j];
          Ak[k] = volr[i] * dzc[j] * kKappa;
        }
      const double *srcs[3] = {gR, gZ, Ak};
      const double *dsts[3] = {b.L.gR, b.L.gZ, b.L.Ak};
      for (int a = 0; a < 3 && rc == MG_OK; ++a)
        if (cudaMemcpy((void *)dsts[a], srcs[a], b.nodes * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
          rc = fail(s, MG_ECUDA, "conductance copy");
      if (p->precision == MG_MIXED && rc == MG_OK) {
        std::vector<float> nf(3 * b.nodes);
        for (size_t k = 0; k < b.nodes; ++k) {
          nf[k] = (float)gR[k];
          nf[b.nodes + k] = (float)gZ[k];
          nf[2 * b.nodes + k] = (float)(Ak[k] * p->n0);
        }
        const float *dst32[3] = {b.M.gR, b.M.gZ, b.M.Ak};
        for (int a = 0; a < 3 && rc == MG_OK; ++a)
          if (cudaMemcpy((void *)dst32[a], nf.data() + a * b.nodes, b.nodes * sizeof(float), cudaMemcpyHostToDevice) !=
              cudaSuccess)
            rc = fail(s, MG_ECUDA, "conductance copy (FP32)");
      }
    }
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) rc = fail(s, MG_ECUDA, "geometry sync");
  }
  s->tr.mu_e = p->mu_e / p->pressure_factor; s->tr.D_e = p->D_e / p->pressure_factor;
  s->tr.mu_p = p->mu_p / p->pressure_factor; s->tr.D_p = p->D_p / p->pressure_factor;
  s->tr.inv_pf = 1.0 / p->pressure_factor;
  s->tr.table = nullptr; s->tr.rows = 0; s->tr.inv_dE = nullptr;
  if (p->table && rc == MG_OK) {
    // the table, then the reciprocal width of each |E| interval (the lookup multiplies by it)
    const int rows = p->table_rows;
    std::vector<double> t6(s->table_h);
    t6.resize((size_t)rows * 6, 0.0);
    for (int k = 0; k + 1 < rows; ++k) t6[(size_t)rows * 5 + k] = 1.0 / (s->table_h[5 * (k + 1)] - s->table_h[5 * k]);
    if (cudaMemcpy(s->table_d, t6.data(), t6.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
      rc = fail(s, MG_ECUDA, "table copy");
    s->tr.table = s->table_d; s->tr.rows = rows; s->tr.inv_dE = s->table_d + (size_t)rows * 5;
  }
  if (rc == MG_OK) {
    // initial state: n = 0, V linear in z; old level = state
    std::vector<double> V((size_t)(g->nz + 1) * (g->nr + 1));
    for (int j = 0; j <= g->nz; ++j)
      for (int i = 0; i <= g->nr; ++i)
        V[(size_t)j * (g->nr + 1) + i] =
            p->V_cathode + (p->V_anode - p->V_cathode) * (g->z[j] - g->z[0]) / (g->z[g->nz] - g->z[0]);
    rc = copy_in(s, s->lv[0], s->lv[0].sv.u[NV], V.data(), MG_HOST, 0, g->nz);
    if (rc == MG_OK && launch_dirichlet(s->lv[0].L, s->lv[0].sv, p->V_cathode, p->V_anode, s->stream) != cudaSuccess)
      rc = fail(s, MG_ECUDA, "dirichlet");
    if (rc == MG_OK) copy_state_async(s, 0, true);
    if (rc == MG_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = fail(s, MG_ECUDA, "init sync");
  }
  if (rc == MG_OK) rc = upload_level_set(s);
  if (rc == MG_OK) rc = setup_coarse_kernel(s);
  if (rc != MG_OK) {
    mg_destroy(s);
    return rc;
  }
  *out = s;
  return MG_OK;
}

void mg_destroy(mg_state *s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  else cudaDeviceSynchronize();
  for (cudaEvent_t e : s->prof_ev) cudaEventDestroy(e);
  for (int l = 0; l < kMaxLevels; ++l)
    if (s->vexec[l]) cudaGraphExecDestroy(s->vexec[l]);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  if (s->hctl) cudaFreeHost(s->hctl);
  if (s->owns_ws && s->ws) cudaFree(s->ws);
  if (s->hout) cudaFreeHost(s->hout);
  if (s->bprog) cudaFree(s->bprog);
  for (int l = 0; l < kMaxLevels; ++l) {
    if (s->bcs64[l]) cudaFree(s->bcs64[l]);
    if (s->bcs32[l]) cudaFree(s->bcs32[l]);
  }
  delete s;
}

const char *mg_last_error(const mg_state *s) { return s ? s->err.c_str() : "null state"; }

int mg_set_state(mg_state *s, const double *ne, const double *np, const double *V, int where) {
  if (!s || !ne || !np || !V) return MG_EINVAL;
  int rc = check_where(s, where);
  if (rc) return rc;
  LevelBuf &b = s->lv[0];
  const double *src[3] = {ne, np, V};
  for (int q = 0; q < 3; ++q)
    if ((rc = copy_in(s, b, b.sv.u[q], src[q], where, 0, b.nz))) return rc;
  CK(launch_dirichlet(b.L, b.sv, s->prm.V_cathode, s->prm.V_anode, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return MG_OK;
}

int mg_set_old_state(mg_state *s, const double *ne, const double *np, const double *V, int where) {
  if (!s || !ne || !np || !V) return MG_EINVAL;
  int rc = check_where(s, where);
  if (rc) return rc;
  LevelBuf &b = s->lv[0];
  const double *src[3] = {ne, np, V};
  for (int q = 0; q < 3; ++q)
    if ((rc = copy_in(s, b, b.sv.uold[q], src[q], where, 0, b.nz))) return rc;
  CK(cudaStreamSynchronize(s->stream));
  return MG_OK;
}

int mg_get_state(const mg_state *cs, double *ne, double *np, double *V, int where) {
  mg_state *s = const_cast<mg_state *>(cs);
  if (!s || !ne || !np || !V) return MG_EINVAL;
  int rc = check_where(s, where);
  if (rc) return rc;
  LevelBuf &b = s->lv[0];
  double *dst[3] = {ne, np, V};
  for (int q = 0; q < 3; ++q)
    if ((rc = copy_out(s, b, dst[q], b.sv.u[q], where))) return rc;
  CK(cudaStreamSynchronize(s->stream));
  return MG_OK;
}

int mg_set_sources(mg_state *s, const double *S_e, const double *S_p, int where) {
  if (!s || !S_e || !S_p) return MG_EINVAL;
  int rc = check_where(s, where);
  if (rc) return rc;
  LevelBuf &b = s->lv[0];
  if ((rc = copy_in(s, b, (double *)b.sv.S[0], S_e, where, 0, b.nz))) return rc;
  if ((rc = copy_in(s, b, (double *)b.sv.S[1], S_p, where, 0, b.nz))) return rc;
  CK(cudaStreamSynchronize(s->stream));
  return MG_OK;
}

int mg_residual(mg_state *s, double dt, double *F_ne, double *F_np, double *F_V, double rho[3], int where) {
  if (!s) return MG_EINVAL;
  int rc = check_where(s, where);
  if (rc) return rc;
  LevelBuf &b = s->lv[0];
  double *Fo[3] = {b.L.r[0], b.L.r[1], b.L.r[2]};
  double rh[3];
  if ((rc = residual(s, 0, dt, false, Fo, rh, nullptr))) return rc;
  if (rho) for (int q = 0; q < 3; ++q) rho[q] = rh[q];
  double *dst[3] = {F_ne, F_np, F_V};
  for (int q = 0; q < 3; ++q)
    if (dst[q] && (rc = copy_out(s, b, dst[q], b.L.r[q], where))) return rc;
  CK(cudaStreamSynchronize(s->stream));
  return MG_OK;
}

int mg_jacobian_apply(mg_state *s, double dt, const double *v_ne, const double *v_np, const double *v_V,
                      double *o_ne, double *o_np, double *o_V, int where) {
  if (!s || !v_ne || !v_np || !v_V || !o_ne || !o_np || !o_V) return MG_EINVAL;
  int rc = check_where(s, where);
  if (rc) return rc;
  LevelBuf &b = s->lv[0];
  CK(launch_coef(b.L, b.sv, s->tr, s->stream));
  CK(launch_factor(b.L, nullptr, dt, s->prm.n0, s->stream));
  const double *src[3] = {v_ne, v_np, v_V};
  // caller rows -> the residual scratch -> du (colour-split); a Dirichlet wall carries no
  // unknowns, so its entries of v are zeroed and do not enter J v
  for (int q = 0; q < 3; ++q)
    if ((rc = copy_in(s, b, b.L.r[q], src[q], where, 1, b.nz - 1))) return rc;
  CK(launch_zero_du<double>(b.L, s->stream));
  CK(launch_split_rows(b.L, b.L.r, b.L.du, s->stream));
  // J v is written on the unknown rows and columns only: the rest of the output is zero
  for (int q = 0; q < 3; ++q) CK(cudaMemsetAsync(b.L.r[q], 0, b.nodes * sizeof(double), s->stream));
  CK(launch_linres<double>(b.L, b.L.du, nullptr, b.L.r, nullptr, nullptr, nullptr, s->stream));
  // full_jacobian: add the field dependence of mu, D
  if (s->prm.full_jacobian) CK(launch_add_transport(b.L, b.sv, s->tr, b.L.du[NV], b.L.r, s->stream));
  double *dst[3] = {o_ne, o_np, o_V};
  for (int q = 0; q < 3; ++q)
    if ((rc = copy_out(s, b, dst[q], b.L.r[q], where))) return rc;
  CK(cudaStreamSynchronize(s->stream));
  return MG_OK;
}

int mg_linear_solve(mg_state *s, double dt, const double *f_ne, const double *f_np, const double *f_V,
                    double *x_ne, double *x_np, double *x_V, double eta, int max_cycles, double *history,
                    int *cycles, int where) {
  if (!s || !f_ne || !f_np || !f_V || !x_ne || !x_np || !x_V || max_cycles < 0) return MG_EINVAL;
  int rc = check_where(s, where);
  if (rc) return rc;
  LevelBuf &b = s->lv[0];
  double tn[3];
  if ((rc = residual(s, 0, dt, false, nullptr, nullptr, tn))) return rc;
  if ((rc = build_hierarchy(s, 0, dt))) return rc;
  const double *src[3] = {f_ne, f_np, f_V};
  // caller rows -> the residual scratch (row layout) -> f (colour-split layout)
  for (int q = 0; q < 3; ++q)
    if ((rc = copy_in(s, b, b.L.r[q], src[q], where, 1, b.nz - 1))) return rc;
  CK(launch_split_rows(b.L, b.L.r, b.L.f, s->stream));
  for (int q = 0; q < 3; ++q) CK(cudaMemsetAsync(b.L.r[q], 0, b.nodes * sizeof(double), s->stream));
  int nc = 0;
  bool ok;
  if ((rc = linear_solve(s, 0, eta, max_cycles, tn, history, &nc, &ok))) return rc;
  if (cycles) *cycles = nc;
  double *dst[3] = {x_ne, x_np, x_V};
  CK(launch_join_rows(b.L, b.L.du, b.L.r, s->stream));
  for (int q = 0; q < 3; ++q)
    if ((rc = copy_out(s, b, dst[q], b.L.r[q], where))) return rc;
  CK(cudaStreamSynchronize(s->stream));
  return ok ? MG_OK : fail(s, MG_ENOCONV, "linear solve: tolerance not reached in %d V-cycles", nc);
}

int mg_step(mg_state *s, double dt, double tol, mg_stats *st) {
  if (!s || !(dt > 0.0) || !(tol > 0.0)) return MG_EINVAL;
  int newton = 0;
  int rc = step(s, 0, dt, tol, &newton);
  if (rc == MG_OK) { s->stats.steps_accepted++; s->stats.sim_time += dt; }
  else if (rc != MG_ECUDA) s->stats.steps_rejected++;
  s->stats.dt_last = dt;
  if (st) *st = s->stats;
  if (rc == MG_ENOCONV) fail(s, rc, "step rejected (Newton cap, linear solve or correction limit)");
  if (rc == MG_ENONFINITE) fail(s, rc, "step rejected (non-finite values)");
  return rc;
}

int mg_march(mg_state *s, double dt_start, double tol, mg_stats *st) {
  if (!s || !(dt_start > 0.0) || !(tol > 0.0)) return MG_EINVAL;
  int rc = march(s, 0, dt_start, tol);
  if (st) *st = s->stats;
  return rc;
}

// Multilevel continuation (abstract and Sec. 2): steady state on level `from` (state and
// sources injected from the finest level, march from dt1), then on each finer level the
// prolonged steady state and a march from dt_max.  The coarse_* statistics count every level
// but the finest.
int mg_solve_steady(mg_state *s, double tol, mg_stats *st) {
  if (!s || !(tol > 0.0)) return MG_EINVAL;
  if (s->nlev < 2) return fail(s, MG_EINVAL, "continuation needs at least two grid levels");
  const int from = s->prm.chain_from;
  if (from < 1 || from >= s->nlev)
    return fail(s, MG_EINVAL, "chain_from = %d outside 1 .. %d", from, s->nlev - 1);
  for (int l = 1; l <= from; ++l)
    CK(launch_inject(s->lv[l - 1].L, s->lv[l - 1].sv, s->lv[l].L, s->lv[l].sv, false, true, s->stream));
  const mg_stats before = s->stats;
  auto count_coarse = [&]() {
    s->stats.coarse_steps += s->stats.steps_accepted + s->stats.steps_rejected - before.steps_accepted -
                             before.steps_rejected;
    s->stats.coarse_newton += s->stats.newton_iterations - before.newton_iterations;
    s->stats.coarse_vcycles += s->stats.vcycles - before.vcycles;
  };
  int rc = march(s, from, s->prm.dt1, tol);
  bool counted = false;
  for (int l = from - 1; l >= 0 && rc == MG_OK; --l) {
    if (l == 0) { count_coarse(); counted = true; }
    LevelBuf &f = s->lv[l], &c = s->lv[l + 1];
    CK(launch_prolong_state(c.L, c.sv, f.L, f.sv, s->stream));
    CK(launch_dirichlet(f.L, f.sv, s->prm.V_cathode, s->prm.V_anode, s->stream));
    rc = march(s, l, s->prm.dt_max, tol);
  }
  if (!counted) count_coarse();
  if (st) *st = s->stats;
  return rc;
}

int mg_solve_steady_guess(mg_state *s, const double *ne, const double *np, const double *V, int where, double tol,
                          mg_stats *st, int *used_fallback) {
  if (!s || !ne || !np || !V || !(tol > 0.0)) return MG_EINVAL;
  int rc = check_where(s, where);
  if (rc) return rc;
  if (used_fallback) *used_fallback = 0;
  LevelBuf &b = s->lv[0];
  for (int q = 0; q < 3; ++q)
    CK(cudaMemcpyAsync(b.ubak[q], b.sv.u[q], b.nodes * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
  const double *src[3] = {ne, np, V};
  for (int q = 0; q < 3; ++q)
    if ((rc = copy_in(s, b, b.sv.u[q], src[q], where, 0, b.nz))) return rc;
  CK(launch_dirichlet(b.L, b.sv, s->prm.V_cathode, s->prm.V_anode, s->stream));
  // march from the guess with the long step; a march that needs more than kGuessSteps steps or
  // fails counts as divergence, and the continuation from the saved state takes over
  constexpr int kGuessSteps = 60;
  const int saved = s->prm.max_steps;
  const double saved_dt = s->prm.dt_max;
  s->prm.max_steps = std::min(saved, kGuessSteps);
  s->prm.dt_max = std::max(saved_dt, s->prm.guess_dt_max);
  if (s->prm.guess_level == 1 && s->nlev >= 2) {
    // the guess replaces the initial state of the coarse march (long step from the start),
    // then the continuation proceeds as usual
    LevelBuf &c = s->lv[1];
    CK(launch_inject(b.L, b.sv, c.L, c.sv, false, true, s->stream));
    rc = march(s, 1, std::min(saved_dt, s->prm.guess_dt_start), tol);
    if (rc == MG_OK) {
      CK(launch_prolong_state(c.L, c.sv, b.L, b.sv, s->stream));
      CK(launch_dirichlet(b.L, b.sv, s->prm.V_cathode, s->prm.V_anode, s->stream));
      rc = march(s, 0, saved_dt, tol);
    }
  } else {
    rc = march(s, 0, std::min(saved_dt, s->prm.guess_dt_start), tol);
  }
  s->prm.max_steps = saved;
  s->prm.dt_max = saved_dt;
  if (rc == MG_ECUDA) return rc;
  if (rc != MG_OK) {
    for (int q = 0; q < 3; ++q)
      CK(cudaMemcpyAsync(b.sv.u[q], b.ubak[q], b.nodes * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
    if (used_fallback) *used_fallback = 1;
    rc = mg_solve_steady(s, tol, nullptr);
  }
  if (st) *st = s->stats;
  return rc;
}

int mg_get_stats(const mg_state *s, mg_stats *out) {
  if (!s || !out) return MG_EINVAL;
  *out = s->stats;
  return MG_OK;
}

void mg_reset_stats(mg_state *s) {
  if (s) std::memset(&s->stats, 0, sizeof(s->stats));
}

uint64_t mg_kernel_launches(void) { return (uint64_t)total_launches(); }

int mg_profile_begin(mg_state *s, int kernel, int level) {
  if (!s || kernel < MG_PROF_SMOOTH || kernel > MG_PROF_COARSE_FACTOR || level < 0 || level >= s->nlev)
    return fail(s, MG_EINVAL, "mg_profile_begin: bad kernel or level");
  if (s->prof_ev.empty()) {
    s->prof_ev.resize(2 * kProfMax);
    for (auto &e : s->prof_ev) CK(cudaEventCreate(&e));
  }
  CK(cudaStreamSynchronize(s->stream));
  s->prof_kernel = kernel;
  s->prof_level = level;
  s->prof_n = 0;
  return MG_OK;
}

int mg_profile_end(mg_state *s, int64_t *launches, double *total_ms) {
  if (!s) return MG_EINVAL;
  CK(cudaStreamSynchronize(s->stream));
  double tot = 0.0;
  for (int k = 0; k < s->prof_n; ++k) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, s->prof_ev[2 * k], s->prof_ev[2 * k + 1]));
    tot += ms;
  }
  if (launches) *launches = s->prof_n;
  if (total_ms) *total_ms = tot;
  s->prof_kernel = 0;
  s->prof_level = -1;
  s->prof_n = 0;
  return MG_OK;
}

double mg_probe_fp64_gflops(void *stream) { return probe_fp64_gflops((cudaStream_t)stream); }

int mg_time_smoother(mg_state *s, int level, int precision, int sweeps, double *us_per_launch,
                     int *launches_per_sweep) {
  if (!s || !us_per_launch || level < 0 || level >= s->nlev - 1 || (precision != 0 && precision != 1) ||
      (precision == 1 && !mixed(s)) || sweeps < 1 || sweeps > 4096)
    return fail(s, MG_EINVAL, "mg_time_smoother: bad level, precision or sweep count");
  cudaStream_t st = s->stream, cs = s->cap_stream;
  // the sweeps, as a V-cycle issues them, captured into one graph on the private capture
  // stream and replayed on the state's stream; only the level's correction buffers are
  // written, and they are zeroed afterwards
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  CK(cudaStreamSynchronize(st));
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  set_capturing(true);
  const int rc = precision == 0 ? smooth_sweeps<double>(s, level, sweeps, cs) : smooth_sweeps<float>(s, level, sweeps, cs);
  const int64_t launches = captured_launches();
  set_capturing(false);
  const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
  if (rc != MG_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
  CK(ec);
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  CK(e);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float ms = 0.f;
  e = cudaGraphLaunch(exec, st);                 // warm-up replay
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGraphExecDestroy(exec);
  CK(e);
  if (precision == 0) CK(launch_zero_du<double>(s->lv[level].L, st));
  else CK(launch_zero_du<float>(s->lv[level].M, st));
  CK(cudaStreamSynchronize(st));
  *us_per_launch = launches > 0 ? 1000.0 * ms / (double)launches : 0.0;
  if (launches_per_sweep) *launches_per_sweep = (int)(launches / sweeps);
  return MG_OK;
}


int mg_autotune(mg_state *s, int32_t *shapes_out) {
  if (!s) return MG_EINVAL;
  // half-sweep blocks (bx * by threads over the colour's nodes) of at most 128 threads: on the
  // small levels larger blocks leave most SMs idle (256 threads on 129^2: 11 % slower steady
  // solves), and they never won on 257^2
  static const int cand[][2] = {{32, 1}, {64, 1}, {128, 1}};
  // the tuning launches write only the correction buffers du and du2 of each level
  const int nc = (int)(sizeof(cand) / sizeof(cand[0]));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int rc = MG_OK;
  // the smoother only rewrites the correction arrays, so tuning leaves the state untouched
  for (int l = 0; l < s->nlev - 1 && rc == MG_OK; ++l) {
    for (int prec = 0; prec < (mixed(s) ? 2 : 1) && rc == MG_OK; ++prec) {
      float best = 1e30f;
      int bi = 1;
      for (int c = 0; c < nc && rc == MG_OK; ++c) {
        float ms = 0.f;
        rc = prec == 0 ? time_shape<double>(s, l, cand[c][0], cand[c][1], 20, e0, e1, &ms)
                       : time_shape<float>(s, l, cand[c][0], cand[c][1], 20, e0, e1, &ms);
        if (ms < best) { best = ms; bi = c; }
      }
      LevelBuf &b = s->lv[l];
      if (prec == 0) { b.sbx = cand[bi][0]; b.sby = cand[bi][1]; }
      else { b.sbx32 = cand[bi][0]; b.sby32 = cand[bi][1]; }
      // fused-sweep tile shape
      float bestf = 1e30f;
      int bf = 1;
      for (int c = 0; c < kSweepShapes && rc == MG_OK; ++c) {
        float ms = 0.f;
        rc = prec == 0 ? time_sweep<double>(s, l, c, 10, e0, e1, &ms) : time_sweep<float>(s, l, c, 10, e0, e1, &ms);
        if (ms < bestf) { bestf = ms; bf = c; }
      }
      if (prec == 0) b.sw = bf; else b.sw32 = bf;
      // FP32: keep the fused sweep only where it beats two half sweeps of the best shape by
      // more than the timing noise (3 %), so that near-ties give the same choice run after run.
      // FP64: never.  Back-to-back launches of one kernel favour the fused sweep, but inside the
      // V-cycle its red ring recompute costs FP64 work that two half sweeps do not: on the 257^2
      // steady solve every FP64 level ran as fast or faster with half sweeps (129^2: 5 % of the
      // solve), while the FP32 choices were within noise of each other.
      const int fz = (prec == 1 && bestf < 0.97f * 2.0f * best) ? 1 : 0;
      if (prec == 0) b.fuse = fz; else b.fuse32 = fz;
      if (shapes_out) {
        shapes_out[6 * l + 3 * prec] = cand[bi][0];
        shapes_out[6 * l + 3 * prec + 1] = cand[bi][1];
        shapes_out[6 * l + 3 * prec + 2] = fz;
      }

    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // graphs recorded the old launch shapes
  for (int l = 0; l < kMaxLevels; ++l)
    if (s->vexec[l]) { cudaGraphExecDestroy(s->vexec[l]); s->vexec[l] = nullptr; }
  CK(launch_zero_du<double>(s->lv[0].L, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return rc;
}

int mg_set_smoother(mg_state *s, int level, int precision, int bx, int by, int fused, int tile) {
  if (!s) return MG_EINVAL;
  if (level < 0 || level >= s->nlev || (precision != 0 && precision != 1) || (fused != 0 && fused != 1))
    return fail(s, MG_EINVAL, "mg_set_smoother: bad level / precision / fused flag");
  if ((bx != 32 && bx != 64 && bx != 128) || by < 1 || bx * by > 256 || tile < 0 || tile >= kSweepShapes)
    return fail(s, MG_EINVAL, "mg_set_smoother: bad block (%d, %d) or tile %d", bx, by, tile);
  LevelBuf &b = s->lv[level];
  if (precision == 0) { b.sbx = bx; b.sby = by; b.fuse = fused; b.sw = tile; }
  else { b.sbx32 = bx; b.sby32 = by; b.fuse32 = fused; b.sw32 = tile; }
  // graphs recorded the old launch shapes
  for (int l = 0; l < kMaxLevels; ++l)
    if (s->vexec[l]) { cudaGraphExecDestroy(s->vexec[l]); s->vexec[l] = nullptr; }
  return MG_OK;
}

int mg_set_level_sweeps(mg_state *s, int level, int nu1, int nu2) {
  if (!s) return MG_EINVAL;
  if (level < 0 || level >= s->nlev || nu1 < -1 || nu2 < -1 || (nu1 >= 0) != (nu2 >= 0) ||
      (nu1 >= 0 && nu1 + nu2 < 1))
    return fail(s, MG_EINVAL, "mg_set_level_sweeps: bad level %d or sweeps (%d, %d)", level, nu1, nu2);
  s->lv[level].nu1 = nu1;
  s->lv[level].nu2 = nu2;
  for (int l = 0; l < kMaxLevels; ++l)
    if (s->vexec[l]) { cudaGraphExecDestroy(s->vexec[l]); s->vexec[l] = nullptr; }
  return setup_coarse_kernel(s);  // the coarse-cycle kernel carries its levels' sweep counts
}

int mg_num_levels(const mg_state *s) { return s ? s->nlev : 0; }

// ---------------------------------------------------------------- batched steady solves
namespace {
// The persistent form: every discharge's whole steady solve in one launch of the work-list
// kernel, replayed from a captured graph (descriptors in, the launch, descriptors back).
// ms_out[k]: from the launch's start to discharge k's solve ending (device clock).
int solve_batch_persistent(mg_state **states, int n, double tol, double *ms_out, int *rc_out) {
  int rc = MG_OK;
  for (int k = 0; k < n && rc == MG_OK; ++k) {
    rc = build_batch_program(states[k]);
    if (rc == MG_OK && cudaStreamSynchronize(states[k]->stream) != cudaSuccess) rc = MG_ECUDA;
  }
  if (rc != MG_OK) return rc;
  const int grid = batch_grid();
  if (grid <= 0) return MG_ECUDA;
  cudaStream_t st = nullptr;
  BatchHead *d_head = nullptr, *h_head = nullptr;
  BatchInst *d_inst = nullptr, *h_inst = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  auto cleanup = [&]() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (st) cudaStreamDestroy(st);
    cudaFree(d_head);
    cudaFree(d_inst);
    cudaFreeHost(h_head);
    cudaFreeHost(h_inst);
  };
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&d_head, sizeof(BatchHead)) != cudaSuccess || cudaMalloc(&d_inst, n * sizeof(BatchInst)) != cudaSuccess ||
      cudaMallocHost(&h_head, sizeof(BatchHead)) != cudaSuccess ||
      cudaMallocHost(&h_inst, n * sizeof(BatchInst)) != cudaSuccess) {
    cleanup();
    return MG_ECUDA;
  }
  // largest discharges first: the CTAs look for work in this order (longest chains first)
  std::vector<int> order(n);
  for (int k = 0; k < n; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return states[a]->lv[0].nodes > states[b]->lv[0].nodes; });
  for (int k = 0; k < n; ++k) batch_describe(states[order[k]], tol, h_inst[k]);
  std::memset(h_head, 0, sizeof(BatchHead));
  h_head->n = n;
  h_head->t0 = ~0ull;
  set_capturing(true);
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaMemcpyAsync(d_head, h_head, sizeof(BatchHead), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_inst, h_inst, n * sizeof(BatchInst), cudaMemcpyHostToDevice, st);
    launch_batch(d_head, d_inst, grid, st);
    cudaMemcpyAsync(h_inst, d_inst, n * sizeof(BatchInst), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(h_head, d_head, sizeof(BatchHead), cudaMemcpyDeviceToHost, st);
    e = cudaStreamEndCapture(st, &graph);
  }
  set_capturing(false);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  count_launch(1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return MG_ECUDA;
  }
  const bool gave_up = h_head->err != 0u || h_head->ndone != n;
  int first = MG_OK;
  for (int j = 0; j < n; ++j) {
    const int k = order[j];
    mg_state *s = states[k];
    const BatchInst &I = h_inst[j];
    int r = I.m.rc;
    if (gave_up) {
      r = MG_ETIMEOUT;
      fail(s, r, "batched solve: the device work list stopped making progress");
    } else {
      batch_collect(s, I);
      if (r != MG_OK) fail(s, r, "march: steady residual not reached in %d steps", s->prm.max_steps);
    }
    if (rc_out) rc_out[k] = r;
    if (ms_out) ms_out[k] = I.m.t_done > h_head->t0 ? (double)(I.m.t_done - h_head->t0) * 1e-6 : 0.0;
    if (first == MG_OK && r != MG_OK) first = r;
  }
  cleanup();
  return first;
}
}  // namespace

int mg_solve_steady_batch(mg_state **states, int n, double tol, int workers, double *ms_out, int *rc_out) {
  if (n < 0 || !(tol > 0.0) || workers < 0 || (n > 0 && !states)) return MG_EINVAL;
  if (n == 0) return MG_OK;
  for (int k = 0; k < n; ++k)
    if (!states[k]) return MG_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MG_ECUDA;
  if (workers == 0) {
    bool all = true;
    for (int k = 0; k < n; ++k) all = all && batchable(states[k]);
    if (all) return solve_batch_persistent(states, n, tol, ms_out, rc_out);
    workers = 16;  // a configuration the persistent launch does not cover: host threads
  }
  workers = std::max(1, std::min(workers, n));
  std::atomic<int> next(0);
  std::vector<int> rcs(n, MG_OK);
  auto work = [&]() {
    cudaSetDevice(dev);
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= n) break;
      const auto t0 = std::chrono::steady_clock::now();
      int rc = mg_solve_steady(states[k], tol, nullptr);
      if (cudaStreamSynchronize(states[k]->stream) != cudaSuccess && rc == MG_OK) rc = MG_ECUDA;
      const auto t1 = std::chrono::steady_clock::now();
      rcs[k] = rc;
      if (ms_out) ms_out[k] = std::chrono::duration<double, std::milli>(t1 - t0).count();
    }
  };
  std::vector<std::thread> pool;
  for (int w = 1; w < workers; ++w) pool.emplace_back(work);
  work();
  for (auto &t : pool) t.join();
  int first = MG_OK;
  for (int k = 0; k < n; ++k) {
    if (rc_out) rc_out[k] = rcs[k];
    if (first == MG_OK && rcs[k] != MG_OK) first = rcs[k];
  }
  return first;
}

int mg_autotune_batch(mg_state **states, int n, double tol, int *grain_out) {
  if (!states || n <= 0 || !(tol > 0.0)) return MG_EINVAL;
  for (int k = 0; k < n; ++k)
    if (!states[k] || !batchable(states[k])) return MG_EINVAL;
  // every trial starts from the states as they are now: solution (finest level), statistics and
  // start data saved here and restored before each trial and at the end
  std::vector<mg_stats> st0(n);
  std::vector<std::vector<double>> ss0(n);
  std::vector<bool> sv0(n);
  for (int k = 0; k < n; ++k) {
    mg_state *s = states[k];
    LevelBuf &b = s->lv[0];
    for (int q = 0; q < 3; ++q)
      if (cudaMemcpyAsync(b.ubak[q], b.sv.u[q], b.nodes * sizeof(double), cudaMemcpyDeviceToDevice, s->stream) !=
          cudaSuccess)
        return MG_ECUDA;
    st0[k] = s->stats;
    ss0[k].assign(s->start_sums, s->start_sums + 16);
    sv0[k] = s->start_valid;
  }
  auto restore = [&]() -> int {
    for (int k = 0; k < n; ++k) {
      mg_state *s = states[k];
      LevelBuf &b = s->lv[0];
      for (int q = 0; q < 3; ++q)
        if (cudaMemcpyAsync(b.sv.u[q], b.ubak[q], b.nodes * sizeof(double), cudaMemcpyDeviceToDevice, s->stream) !=
            cudaSuccess)
          return MG_ECUDA;
      if (cudaStreamSynchronize(s->stream) != cudaSuccess) return MG_ECUDA;
      s->stats = st0[k];
      std::copy(ss0[k].begin(), ss0[k].end(), s->start_sums);
      s->start_valid = sv0[k];
    }
    return MG_OK;
  };
  auto set_shape = [&](int g, int cn) {
    for (int k = 0; k < n; ++k) {
      mg_state *s = states[k];
      if ((s->bgrain != g || s->bcoarse_n != cn) && s->bprog) {
        cudaFree(s->bprog);
        s->bprog = nullptr;
      }
      s->bgrain = g;
      s->bcoarse_n = cn;
    }
  };
  static const int kGrains[] = {2, 4, 8};
  static const int kCoarse[] = {16, 32, 64};
  int best = 4, best_c = 16, rc = MG_OK;
  double best_ms = 1e300;
  for (int cn : kCoarse)
    for (int g : kGrains) {
      if ((rc = restore())) return rc;
      set_shape(g, cn);
      const auto t0 = std::chrono::steady_clock::now();
      rc = solve_batch_persistent(states, n, tol, nullptr, nullptr);
      const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      if (rc != MG_OK) break;
      if (ms < best_ms) { best_ms = ms; best = g; best_c = cn; }
    }
  const int rc2 = restore();
  set_shape(best, best_c);
  if (grain_out) *grain_out = best + 100 * best_c;
  return rc != MG_OK ? rc : rc2;
}

}  // extern "C"
