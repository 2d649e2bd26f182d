// Internal declarations of the GB300 multigrid solver (not part of the C ABI).
//
// Storage: every node field is a (nz + 1) x P array (P = pitch >= nr + 1, a
// multiple of 4 so that each row starts on a 32-byte boundary), row j (axial)
// slow, column i (radial) fast.  Face coefficients are stored at the node that
// is the lower-index end of the face: r-face (i+1/2, j) at [j][i], z-face
// (i, j+1/2) at [j][i].
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mgk {

// Physical constants (SI): e / eps0 of eq. 5.
constexpr double kECharge = 1.602176634e-19;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kKappa = kECharge / kEps0;

enum { NE = 0, NP = 1, NV = 2 };
// kernel kinds that may use programmatic dependent launch (mg_params.pdl bits)
enum { PDL_SMOOTH = 1, PDL_TRANSFER = 2, PDL_NORM = 4, PDL_COARSE = 8, PDL_OTHER = 16, PDL_ALL = 31 };
// face-coefficient slots: per species s (0 = electrons, 1 = ions): G-term, F-term, V-derivative
enum { CGE = 0, CFE = 1, CVE = 2, CGP = 3, CFP = 4, CVP = 5, NCOEF = 6 };
// per-node factors of the 3x3 diagonal block [[a11, 0, a13], [0, a22, a23], [-ak, ak, a33]]
// (ak = A e/eps0): inverse pivots, Schur-complement multipliers q1 = -ak/a11, q2 = ak/a22,
// inverse Schur complement, and the two couplings to V
enum { FI11 = 0, FI22 = 1, FQ1 = 2, FQ2 = 3, FIS = 4, FA13 = 5, FA23 = 6, NFAC = 7 };
// The factor arrays, the right-hand sides f and the corrections du are stored colour-split
// within each row of pitch P: node (i, j) with i + j even at i / 2, the other colour at P / 2 + i / 2 (P is a
// multiple of 4 and exceeds nr, so both halves hold their row's nodes).  A half sweep then
// reads its colour's factors and right-hand sides and the other colour's corrections as
// contiguous runs per row, and writes its own corrections as one, instead of every other
// element.  Slots past nr stay zero (multiplied by zero face coefficients at i = 0 and nr).
__host__ __device__ __forceinline__ size_t cidx(int P, int i, int j) {
  return (size_t)j * P + (((i + j) & 1) ? (P >> 1) : 0) + (i >> 1);
}
// Colour-split positions of node (i, j) (self) and of its four neighbours, which are all of
// the other colour: E and W are adjacent slots of that colour's half of row j, N and S the
// slot i / 2 of its half of rows j + 1 and j - 1.
struct SplitNb {
  size_t self, E, W, N, S;
};
__host__ __device__ __forceinline__ SplitNb split_nb(int P, int i, int j) {
  const int half = P >> 1, h = i >> 1;
  const int other = ((i + j) & 1) ? 0 : half;          // the other colour's half
  const size_t row = (size_t)j * P;
  SplitNb n;
  n.self = row + (half - other) + h;
  n.E = row + other + h + (i & 1);
  n.W = n.E - 1;
  n.N = row + P + other + h;
  n.S = row - P + other + h;
  return n;
}
enum { DA11 = 0, DA22 = 1, DA33 = 2, NDIA = 3 };

// Transport inputs (mu, D constant or tabulated in |E|), already divided by the pressure factor.
struct Transport {
  double mu_e, D_e, mu_p, D_p;
  const double *table;  // device, rows x 5 (|E|, mu_e, D_e, mu_p, D_p), or nullptr
  int rows;
  double inv_pf;        // 1 / pressure factor (applied to tabulated values)
  const double *inv_dE; // device, 1 / (|E|_{k+1} - |E|_k) per table interval, or nullptr (divide)
};

// One multigrid level: geometry, state and work arrays (device pointers).
template <typename T>
struct LevelT {
  int nr, nz, P;
  int ni;                    // unknown columns: nr + 1, or nr with a Dirichlet wall
  int pdl;                   // host side: PDL_* bits of the kernel kinds launched with programmatic
                             // dependent launch (they start while the previous kernel finishes)
  T dr;
  const T *dz, *dzc, *volr;  // nz, nz+1, nr+1 (geometry in the level's arithmetic type)
  const T *idz;              // 1 / dz (nz entries)
  const T *zf;               // (z_j - z_0) / (z_nz - z_0) (nz + 1 entries; the wall's V profile)
  T idr;                     // 1 / dr
  const T *wz;               // odd fine row j: weight of the upper coarse node (nz+1 entries)
  const T *gR, *gZ, *Ak;     // node arrays: r-face and z-face Poisson conductances, (e/eps0) A
  T *cr[NCOEF], *cz[NCOEF];  // face coefficients
  T *fac[NFAC], *dia[NDIA];  // diagonal-block factors (rebuilt with the coefficients)
  T *du[3], *f[3], *r[3];
  T *du2[3];                 // second correction buffer (ping-pong of the fused sweep)
};
using Level = LevelT<double>;

// The coarse levels handled by one launch of the persistent coarse-cycle kernel (K8).
constexpr int kMaxCoarseSet = 8;
template <typename T>
struct CoarseSet {
  LevelT<T> lv[kMaxCoarseSet];
  int n;                            // levels in the set; the last one is the coarsest
  int nu1[kMaxCoarseSet], nu2[kMaxCoarseSet];  // pre- / post-smoothing sweeps per level
  const double *Minv, *rs, *cs;     // dense inverse of the coarsest level (FP64)
  double nscale;                    // density unit of the view (1 or n0)
};

// Ping-pong correction buffers of one fused red-black sweep (read previous, write next).
template <typename T>
struct SweepIO {
  T *in[3];
  T *out[3];
};
constexpr int kSweepShapes = 6;  // tile shapes of the fused sweep: 32x2 32x4 32x8 64x2 64x4 128x2

struct StateView {           // nonlinear state on one level (FP64)
  double *u[3], *uold[3];
  const double *S[2];
};

// Views of every level in device memory, for the kernels that treat all levels of the
// hierarchy in one launch (blockIdx.z selects the level).
constexpr int kMaxLevelSet = 16;
struct LevelSet {
  LevelT<double> L[kMaxLevelSet];
  LevelT<float> M[kMaxLevelSet];
  StateView sv[kMaxLevelSet];
};

// Device-resident control block of one linear solve (device-side V-cycle loop in a CUDA graph).
constexpr int kMaxHist = 512;
struct SolveCtl {
  double w[3];      // per-field weights (norms of the Newton residual's absolute terms)
  double eta;       // relative tolerance of the weighted residual
  double r0;        // weighted residual at du = 0
  double rel;       // last relative weighted residual
  int max_cycles;
  int ncyc;         // V-cycles run
  double hist[kMaxHist];
};

// ---- batched form: one persistent launch runs the steady solves of many discharges ---------
// Each discharge's solve (the continuation, the Delta-t march with its accept / reject logic,
// the Newton loop of every step) runs as a state machine on the device; its GPU work is a
// sequence of phases from the discharge's program (the launches of the single-discharge path,
// in its order).  A phase is a list of work items (tiles); the CTAs of the launch claim tiles
// of any discharge's current phase, and the CTA that finishes a phase's last tile folds its
// reductions, advances the discharge's state machine and publishes its next phase.
enum BatchKind : int32_t {
  BK_INJECT = 0, BK_COEFL, BK_FACTORL, BK_CFACT, BK_ZERO64, BK_NORM0, BK_ZERO32, BK_HALF64, BK_HALF32,
  BK_RESTR64, BK_RESTR32, BK_COARSE64, BK_COARSE32, BK_PROL64, BK_PROL32, BK_MIXUPD, BK_NORMC, BK_UPDATE,
  BK_COEF0, BK_RESID, BK_INJECT1, BK_COPY, BK_PROLST, BK_DIRI, BK_RET, BK_DONE
};
// BK_RESID variants (arg bits): write f, reduce the steady sums and write the steady -F, use 1/dt
enum { RESID_WRITE_F = 1, RESID_STEADY = 2, RESID_DT = 4 };
// BK_COPY variants (arg): u -> u_old, u_old -> u, steady -F -> f
enum { COPY_TO_OLD = 0, COPY_FROM_OLD = 1, COPY_FSS_TO_F = 2 };
struct BPhase {
  int32_t kind;
  int32_t level;    // the level worked on (the root of a Newton iteration, the fine level of a
                    // transfer, the first of a range)
  int32_t arg;      // colour of a half sweep; last level of a range; variant
  int32_t ntiles;   // work items of the phase
  int32_t grain;    // thread-block rounds per work item
  int32_t nblocks;  // thread blocks of the kernel the phase stands for (reduction partials)
};
constexpr int kBatchThreads = 256;   // threads per CTA of the persistent launch
constexpr int kBatchMaxProg = 4096;  // phases per program (12 bits of a ring entry)
// entry points of the subprograms of one level (program counters)
enum { E_INJECT = 0, E_START_COEF, E_START, E_BEGIN_USE, E_BEGIN_COEF, E_BEGIN, E_NEWTON, E_NLOOP, E_NUPD,
       E_RESTORE, E_PROLONG, E_N };
// Device-resident state of one discharge's steady solve (the host's march / step variables)
struct BatchMarch {
  // parameters
  double tol, dt1, dt_max, dt_growth, ntol, rel, limit, eta_p, Vc, Va;
  int32_t from, max_steps, max_newton, eta_adapt;
  // where the solve is
  int32_t stage, lvl, next_lvl, nstep, it, newton_out, reason, coef_current, start_valid, counted, rc, pad;
  double dt, dt_prev, r_start, step_tol, r_step, eta;
  double rho[3], tn[3], rho_steady[3], cand[16], start_sums[16];
  // statistics of this solve (the host adds them to the state's)
  int32_t steps_accepted, steps_rejected, newton_iterations, vcycles, last_newton;
  int32_t coarse_steps, coarse_newton, coarse_vcycles;
  double srho[3], steady_rho, dt_last, sim_time;
  unsigned long long t_done;         // globaltimer when the solve ended
};
struct BatchInst {
  const BPhase *prog;               // device program (every level's subprograms)
  int32_t ent[kMaxLevelSet][E_N];   // subprogram entries per level
  int32_t last, mixed, max_cycles, pad0;
  const LevelSet *S;
  const CoarseSet<double> *cs64[kMaxLevelSet];   // the coarse part of a V-cycle from level l down
  const CoarseSet<float> *cs32[kMaxLevelSet];    // (one phase on one CTA), by l
  Transport tr;
  double dt_inv, n0, eta, w[3];     // of the current Newton iteration (set by the state machine)
  SolveCtl *ctl;
  double *partials, *dout, *Minv, *rs, *cs;
  int *flag;
  double *fss[3];
  BatchMarch m;
  // run state, reset by the host before the launch
  unsigned long long claim;         // (sequence << 32) | work items claimed of the current phase
  unsigned long long ring[4];       // phase `sequence` at sequence & 3: (sequence << 32) | (pc << 20) | work items
  unsigned int done;                // work items finished of the current phase
  int32_t pad1;
};
struct BatchHead {
  int32_t n;                        // discharges in this launch
  int32_t ndone;                    // discharges whose solve has ended
  unsigned int err;                 // 1: no phase finished anywhere for kBatchIdleNs (the launch gave up)
  unsigned int progress;            // phases finished (the CTAs' idle clocks restart when it moves)
  unsigned long long t0;            // globaltimer at the launch's start (the earliest CTA)
};
cudaError_t launch_batch(BatchHead *head, BatchInst *inst, int grid, cudaStream_t st);
int batch_grid();                   // CTAs of the persistent launch: SMs x resident CTAs per SM (0: error)

// ---- launch wrappers (mg_kernels.cu) ------------------------------------------------------
// All take the stream last and return cudaGetLastError() of the launch.  While a stream capture
// is being recorded (set_capturing(true)) launches are not counted: graph replays are counted
// by the host after they ran.
void count_launch(int n = 1);
void set_capturing(bool on);
int captured_launches();  // launches recorded since set_capturing(true)
cudaError_t launch_solve_init(SolveCtl *ctl, const double *norm3, cudaGraphConditionalHandle h, cudaStream_t st);
cudaError_t launch_solve_check(SolveCtl *ctl, const double *norm3, cudaGraphConditionalHandle h, cudaStream_t st);

cudaError_t launch_coef(const Level &L, const StateView &sv, const Transport &tr, cudaStream_t st);
// Residual rows from the face coefficients of the same state (launch_coef first): F, f = -F and
// the norms as launch_residual, without re-evaluating the Scharfetter-Gummel faces.
cudaError_t launch_resid_coef(const Level &L, const StateView &sv, double dt, bool write_f, bool steady_too,
                              double *Fout[3], double *const fsteady[3], double *partials, unsigned *counter,
                              double *out, cudaStream_t st);
// Hierarchy set-up over levels of the device LevelSet in one launch each (L0 = the level whose
// dimensions size the grid): injection of the state of level l0 into levels l0+1 .. l1, face
// coefficients of levels a .. b, diagonal factors (and, mixed, the FP32 coefficient copies) of
// levels a .. b.
cudaError_t launch_inject_levels(const LevelSet *S, const Level &L0, int l0, int l1, cudaStream_t st);
cudaError_t launch_coef_levels(const LevelSet *S, const Level &La, int a, int b, const Transport &tr,
                               cudaStream_t st);
cudaError_t launch_factor_levels(const LevelSet *S, const Level &La, int a, int b, bool mixed, double dt, double n0,
                                 cudaStream_t st);
// Diagonal-block factors of every unknown node from the FP64 face coefficients at step dt; with
// M non-null also the FP32 copies in n0-scaled unknowns (mixed form).
cudaError_t launch_factor(const Level &L, const LevelT<float> *M, double dt, double n0, cudaStream_t st);
// Residual rows F at the state; writes f = -F into L.f (if write_f) and F into Fout (may be null);
// partial sums of F^2 and T^2 per field reduced to out6[0..5] (F2 e,p,V ; T2 e,p,V).
cudaError_t launch_residual(const Level &L, const StateView &sv, const Transport &tr, double dt,
                            bool write_f, double *Fout[3], double *partials, unsigned *counter,
                            double *out6, cudaStream_t st);
template <typename T>
cudaError_t launch_smooth(const LevelT<T> &L, int color, cudaStream_t st, int bx = 32, int by = 2);
template <typename T>
cudaError_t launch_sweep(const LevelT<T> &L, const SweepIO<T> &io, int shape, cudaStream_t st);
// Coarse part of a V-cycle in one launch of a cluster of `cluster` CTAs (1..8) x `threads`.
// smem_bytes > 0 with cluster == 1: the single-CTA form with every coarse array in shared
// memory (prepare_coarse_smem gives the size, 0 if the set does not fit in `limit` bytes).
template <typename T>
cudaError_t launch_coarse_cycle(const CoarseSet<T> *dev_set, int cluster, int threads, size_t smem_bytes, bool pdl,
                                cudaStream_t st);
template <typename T>
size_t prepare_coarse_smem(const CoarseSet<T> &host_set, size_t limit);
// r = f - J v (or out = J v when f == nullptr); optional per-field norms (sum of squares) -> out3
template <typename T>
cudaError_t launch_linres(const LevelT<T> &L, T *const v[3], T *const f[3], T *out[3], double *partials,
                          unsigned *counter, double *out3, cudaStream_t st);
// r = f - J du on level F and its restriction to C in one launch (r stays on chip)
template <typename T>
cudaError_t launch_linres_restrict(const LevelT<T> &F, const LevelT<T> &C, cudaStream_t st);
template <typename T>
cudaError_t launch_prolong_add(const LevelT<T> &C, const LevelT<T> &F, cudaStream_t st);
cudaError_t launch_inject(const Level &F, const StateView &fs, const Level &C, const StateView &cs,
                          bool with_old, bool with_sources, cudaStream_t st);
cudaError_t launch_prolong_state(const Level &C, const StateView &cs, const Level &F,
                                 const StateView &fs, cudaStream_t st);
// Coarsest level: assemble the dense Jacobian, equilibrate, invert (one CTA).
cudaError_t launch_coarse_factor(const Level &L, double dt, double *M, double *Minv, double *rs,
                                 double *cs, int *flag, cudaStream_t st);
template <typename T>
cudaError_t launch_coarse_solve(const LevelT<T> &L, const double *Minv, const double *rs, const double *cs,
                                double nscale, cudaStream_t st);
// u += du on unknown rows; out2[0] = max |dV|, out2[1] = sum of du^2 (non-finite check)
cudaError_t launch_update(const Level &L, const StateView &sv, double *partials, unsigned *counter,
                          double *out2, cudaStream_t st);
template <typename T>
cudaError_t launch_zero_du(const LevelT<T> &L, cudaStream_t st);
// mixed form
cudaError_t launch_full_defect(const Level &L, const StateView &sv, const Transport &tr, double *const fs[3],
                               double *const d[3], double *partials, unsigned *counter, double *out3, cudaStream_t st);
cudaError_t launch_add_transport(const Level &L, const StateView &sv, const Transport &tr, const double *w,
                                 double *out[3], cudaStream_t st);
template <typename T>
cudaError_t launch_zline(const LevelT<T> &L, int color, T *scr, cudaStream_t st);
// r-line zebra half sweep (rows of one parity; at most kRlineMax unknowns a row)
constexpr int kRlineMax = 512;
template <typename T>
cudaError_t launch_rline(const LevelT<T> &L, int color, cudaStream_t st);
cudaError_t launch_add3(double *const acc[3], double *const x[3], size_t n, cudaStream_t st);
cudaError_t launch_split_rows(const Level &L, double *const in[3], double *const out[3], cudaStream_t st);
cudaError_t launch_join_rows(const Level &L, double *const in[3], double *const out[3], cudaStream_t st);
cudaError_t launch_mixed_update(const Level &L, const LevelT<float> &M, double n0, cudaStream_t st);
cudaError_t launch_outer_residual(const Level &L, const LevelT<float> &M, double n0, double *partials,
                                  unsigned *counter, double *out3, cudaStream_t st);
cudaError_t launch_dirichlet(const Level &L, const StateView &sv, double Vc, double Va, cudaStream_t st);
unsigned long long total_launches();
double probe_fp64_gflops(cudaStream_t st);

}  // namespace mgk
