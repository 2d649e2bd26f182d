/*
 * mg.h - C ABI of the GB300 (sm_103a) multigrid solver for the axisymmetric
 * drift-diffusion + Poisson fluid equations of Ristivojevic & Petrovic,
 * "Multigrid solver for axisymmetrical 2D fluid equations" (arXiv:0811.4446).
 *
 * Problem (Sec. 2 of the paper):
 *   continuity       dn/dt + div(n v) = S             (eqs. 1-2), electrons and ions
 *   fluxes           phi_e = -n_e mu_e E - D_e grad n_e,  phi_p = n_p mu_p E - D_p grad n_p (eqs. 3-4)
 *   Poisson          lap V = -(e/eps0)(n_p - n_e),  E = -grad V                 (eqs. 5-6)
 * on (r, z) in [0, R] x [0, d], azimuthal symmetry, nodes r_i = i R/N_r and a
 * caller-given non-equidistant z_0 < ... < z_Nz.  Discretisation: backward Euler
 * (eq. 7), Scharfetter-Gummel face fluxes (eqs. 8-11; eq. 9 read with the G/F
 * pairing of eq. 8), finite-volume cylindrical Poisson rows (eqs. 12-13).  Each
 * implicit step is solved by Newton-Raphson (eq. 14, 3x3-block five-point
 * Jacobian) whose linear systems are solved by multigrid V-cycles; the steady
 * state is reached by the Delta-t ramp and the coarse-to-fine continuation of
 * Sec. 2 ("multilevel prolongation").
 *
 * Boundary conditions: electrode rows z = z_0 (cathode) and z = z_Nz (anode) are
 * Dirichlet: n_e = n_p = 0, V = V_cathode / V_anode.  Axis r = 0: symmetry.
 * Outer wall r = R: zero normal particle flux and dV/dr = 0.
 *
 * Conventions
 *  - Arrays are node arrays of (N_z + 1) x (N_r + 1) doubles, row-major with the
 *    radial index i fastest: a[j * (N_r + 1) + i].  SI units (m, V, s, m^-3).
 *  - `where` selects the memory space of a caller pointer: MG_HOST (pageable or
 *    pinned host memory) or MG_DEVICE (device memory on the state's GPU).
 *  - Caller arrays are copied in or out and never retained.
 *  - Every call is issued on the stream given to mg_create and returns after the
 *    results it reports are available (calls that return norms or statuses
 *    synchronise that stream).
 *  - Return value: MG_OK or a negative MG_E* code; mg_last_error() gives text.
 *    On any error inside a step the state is left at the last accepted step.
 *  - There is no CPU fallback: every arithmetic step runs in CUDA kernels.
 */
#ifndef PAPER_0811_4446_GB300_MG_H
#define PAPER_0811_4446_GB300_MG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  MG_OK = 0,
  MG_EINVAL = -1,     /* bad sizes or parameters                            */
  MG_ECUDA = -2,      /* a CUDA runtime call failed                         */
  MG_ENOCONV = -3,    /* Newton or multigrid exceeded its iteration caps    */
  MG_EREJECT = -4,    /* Delta-t retries exhausted / step count exhausted   */
  MG_ENONFINITE = -5, /* NaN or Inf appeared in a residual or correction    */
  MG_ETIMEOUT = -6,   /* a bounded device-side wait expired                 */
  MG_ENOMEM = -7      /* workspace too small                                */
};

enum { MG_HOST = 0, MG_DEVICE = 1 };
enum { MG_FP64 = 0, MG_MIXED = 1 };

/* Grid (Sec. 2): N_r, N_z intervals (powers of two, >= 2); radius R; z holds
 * N_z + 1 strictly increasing axial node coordinates (host memory).  The
 * multigrid hierarchy takes every other node, so the coarse grids are nested. */
typedef struct mg_grid {
  int32_t nr, nz;
  double R;
  const double *z;
} mg_grid;

/* Physical inputs and solver knobs.  mu, D in m^2/(V s), m^2/s.  When `table`
 * is non-NULL it holds `table_rows` rows of (|E|, mu_e, D_e, mu_p, D_p) with
 * increasing |E| (host memory); mu and D at a face are then interpolated
 * linearly in the face |E| (clamped at the table ends), the inputs the paper
 * says come "from lookup tables" (Sec. 2).  All mu, D are divided by
 * pressure_factor. */
typedef struct mg_params {
  double V_cathode, V_anode;
  double mu_e, D_e, mu_p, D_p;
  const double *table;
  int32_t table_rows;
  int32_t precision;      /* MG_FP64 or MG_MIXED (FP32 V-cycle in FP64 Newton) */
  double pressure_factor;
  int32_t nu1, nu2;       /* pre/post red-black sweeps per level              */
  int32_t coarsest;       /* stop coarsening at min(N_r, N_z) <= coarsest (2..8)*/
  int32_t max_vcycles;    /* per linear solve                                  */
  int32_t max_newton;     /* per time step (the paper observed < 10)           */
  int32_t max_steps;      /* per march                                         */
  double eta;             /* linear tolerance relative to the Newton residual  */
  double newton_tol;      /* per-step tolerance in a march; 0 -> 0.1 * tol     */
  double corr_limit_frac; /* reject a step if max|dV| > frac * |V_anode - V_cathode| */
  double dt1, dt_growth, dt_max; /* Delta-t ramp of Sec. 2                     */
  double n0;              /* density unit of the FP32 inner cycle (eq. 12's n0), m^-3 */
  int32_t use_graphs;     /* 1: each linear solve is one CUDA-graph launch whose V-cycle loop
                             and stopping test run on the device; 0: host-driven loop */
  int32_t fused_sweep;    /* 1: levels may run one launch per red-black sweep (tiled, both
                             colours) where their choice says so (mg_autotune, mg_set_smoother;
                             by default the FP32 view); 0: one launch per colour everywhere.
                             Same result bit for bit. */
  double guess_dt_max;    /* cap of the Delta-t ramp when marching from a learned guess: the
                             ramp starts at dt_max and grows by dt_growth up to this value */
  int32_t guess_level;    /* 0: march the full grid from the guess; 1: the guess (injected)
                             starts the coarse-grid march of the continuation instead */
  double guess_dt_start;  /* first Delta t of the march from a learned guess (then x dt_growth) */
  int32_t coarse_kernel_n;      /* levels whose larger side has <= this many intervals run as
                                   one persistent cluster launch per V-cycle (0: off) */
  int32_t coarse_kernel_ctas;   /* CTAs of that cluster (1..8) */
  int32_t coarse_kernel_threads;/* threads per CTA (32..1024, multiple of 32) */
  int32_t eta_adapt;      /* 1: Newton iteration k solves to eta_k = max(eta, min(0.1,
                             tol / (2 rho_k))) instead of eta (inexact-Newton forcing term) */
  int32_t nu_coarse_n;    /* levels whose larger side has <= this many intervals smooth with
                             nu_coarse1 / nu_coarse2 sweeps instead of nu1 / nu2 (0: off) */
  int32_t nu_coarse1, nu_coarse2;
  int32_t nu_tiny_n;      /* levels whose larger side has <= this many intervals (a subset of the
                             nu_coarse_n levels) smooth with nu_tiny1 / nu_tiny2 sweeps (0: off) */
  int32_t nu_tiny1, nu_tiny2;
  int32_t chain_from;     /* mg_solve_steady starts its march on level chain_from (the grid
                             coarsened 2^chain_from times; 1 <= chain_from < levels) and goes
                             back up one level at a time: prolongation, then a march from
                             dt_max on each finer level (Sec. 2: finer and finer grids) */
  int32_t pdl;            /* kernel kinds launched with programmatic dependent launch (each starts
                             while its predecessor finishes and fetches constant operator data
                             meanwhile): 1 smoothers, 2 residual-restriction and prolongation,
                             4 cycle norms, 8 the coarse-cycle kernel, 16 the other cycle kernels */
  int32_t wall_dirichlet; /* 0: zero normal flux and dV/dr = 0 on the wall r = R (half-cell rows);
                             1: the argon case of Sec. 3: n_e = n_p = 0 and V linear in z between
                             the electrodes on the wall, which then carries no unknowns */
  double newton_tol_rel;  /* > 0: a march step's Newton tolerance is max(the per-step tolerance,
                             newton_tol_rel x the steady residual at the step's start): steps far
                             from the steady state are solved only as far as they can matter for
                             it (0: off; 0 <= newton_tol_rel < 1) */
  int32_t full_jacobian;  /* 1: Newton with the field dependence of mu(|E|), D(|E|) in the
                             Jacobian (Sec. 2): each Newton step solves the full-Jacobian system by
                             defect correction around the multigrid solve of the Picard Jacobian
                             (eq. 14, mu and D frozen); 0: the Picard Jacobian alone */
  int32_t max_corrections; /* defect corrections per Newton iteration with full_jacobian (1..100);
                             not converged -> the step is rejected like a failed linear solve */
  int32_t line_smoother;  /* 0: point-block red-black Gauss-Seidel; 1: z-line Gauss-Seidel in
                             zebra order (even columns, then odd; each column's block-tridiagonal
                             system solved exactly, robust to strong z-coupling); 2: r-line
                             Gauss-Seidel (even rows, then odd; each row's system along r,
                             robust to strong r-coupling; rows of at most 512 unknowns, i.e.
                             N_r <= 256, or 512 with a Dirichlet wall); 3: alternating lines,
                             each sweep z-lines then r-lines.  On every level (the coarse levels
                             then run as separate launches, no coarse-cycle kernel) */
} mg_params;

/* Per-call statistics. */
typedef struct mg_stats {
  int32_t steps_accepted, steps_rejected;
  int32_t newton_iterations;  /* summed over accepted and rejected steps */
  int32_t vcycles;            /* summed over all linear solves            */
  int32_t last_newton;        /* Newton iterations of the last step       */
  double rho[3];              /* last scale-free residual per field (n_e, n_p, V) */
  double steady_rho;          /* last steady residual (max over fields)  */
  double dt_last;
  double sim_time;            /* accumulated accepted Delta t             */
  int32_t coarse_steps;       /* part of the counts above spent on the coarse grid */
  int32_t coarse_newton;      /* of mg_solve_steady's continuation                 */
  int32_t coarse_vcycles;
} mg_stats;

typedef struct mg_state mg_state;

/* Fill *p with the defaults: mu_e = 30, D_e = 60, mu_p = 0.15, D_p = 0.0038,
 * V_cathode = -200, V_anode = 0, nu1 = nu2 = 4, coarsest = 2, eta = 1e-3,
 * max_newton = 10, max_vcycles = 60, max_steps = 400, dt1 = 1e-9,
 * dt_growth = 5, dt_max = 1e-6, corr_limit_frac = 0.5, precision MG_FP64, n0 = 1e14,
 * use_graphs = 1, fused_sweep = 1, guess_dt_max = 1e-3, guess_level = 0, guess_dt_start = 1e-8,
 * coarse_kernel_n = 16,
 * coarse_kernel_ctas = 1, coarse_kernel_threads = 512, eta_adapt = 1, nu_coarse_n = 64,
 * nu_coarse1 = nu_coarse2 = 2, nu_tiny_n = 8, nu_tiny1 = nu_tiny2 = 1 (V(4,4) smoothing on levels
 * larger than 65^2, V(2,2) from 65^2 to 17^2, V(1,1) from 9^2 down),
 * chain_from = 1 (the two-level 129^2 -> 257^2 continuation), pdl = 9 (smoothers and the coarse-cycle kernel), wall_dirichlet = 0,
 * newton_tol_rel = 0.1, full_jacobian = 0, max_corrections = 20, line_smoother = 0.
 *
 * precision = MG_MIXED: every linear solve of eq. 14 is an FP64 defect-correction loop whose
 * corrections come from FP32 V-cycles (FP32 smoother, residual, restriction, prolongation on
 * FP32 copies of the face coefficients, densities in units of n0); the face coefficients
 * (Bernoulli functions) are evaluated in FP64 and the coarsest level is solved in FP64. */
void mg_params_default(mg_params *p);

/* Bytes of device workspace mg_create needs for this grid and parameters. */
size_t mg_workspace_bytes(const mg_grid *g, const mg_params *p);

/* Create a solver state.  `stream` is a cudaStream_t (NULL = legacy default
 * stream) that the state borrows for all its work.  `workspace` is caller-owned
 * device memory of at least mg_workspace_bytes() bytes (256-byte aligned) that
 * must outlive the state; pass NULL to let the library allocate (and free) it.
 * The state starts from n_e = n_p = 0, V linear in z, sources 0. */
int mg_create(const mg_grid *g, const mg_params *p, void *stream, void *workspace,
              size_t workspace_bytes, mg_state **out);
void mg_destroy(mg_state *s);
const char *mg_last_error(const mg_state *s);

/* Copy the state (n_e, n_p, V) in or out.  mg_set_state overwrites the
 * electrode rows with the Dirichlet values. */
int mg_set_state(mg_state *s, const double *ne, const double *np, const double *V, int where);
int mg_get_state(const mg_state *s, double *ne, double *np, double *V, int where);

/* The time level n^k used by mg_residual / mg_jacobian_apply / mg_linear_solve.
 * mg_step sets it itself from the current state. */
int mg_set_old_state(mg_state *s, const double *ne, const double *np, const double *V, int where);

/* Sources S_e, S_p in m^-3 s^-1 (eqs. 1-2). */
int mg_set_sources(mg_state *s, const double *S_e, const double *S_p, int where);

/* Nonlinear residual rows of eq. 7 + eqs. 12/13 in finite-volume form, at the
 * current state, with time level n^k from mg_set_old_state and step dt
 * (dt <= 0: steady residual, time term dropped).  F (3 node arrays n_e, n_p, V
 * rows, zero on the electrode rows, may be NULL) and rho[3] = ||F_f|| / ||T_f||
 * where T_f sums the absolute values of the terms of each row (may be NULL). */
int mg_residual(mg_state *s, double dt, double *F_ne, double *F_np, double *F_V, double rho[3], int where);

/* Jacobian-vector product (eq. 14) at the current state: out = J v.  v and out
 * are 3 node arrays each (electrode rows of v ignored, of out set to 0).  With
 * full_jacobian = 1 in the state's parameters the product includes the field dependence of
 * mu(|E|), D(|E|) (the full Newton Jacobian); otherwise it is the Picard Jacobian. */
int mg_jacobian_apply(mg_state *s, double dt, const double *v_ne, const double *v_np, const double *v_V,
                      double *o_ne, double *o_np, double *o_V, int where);

/* Solve J x = f (eq. 14) at the current state by V-cycles from x = 0 until the
 * field-weighted residual has dropped by eta (weights: the norms of the
 * nonlinear residual's absolute terms at the current state), or max_cycles.
 * history (may be NULL) receives up to max_cycles + 1 relative residuals;
 * *cycles the number of V-cycles run. */
int mg_linear_solve(mg_state *s, double dt, const double *f_ne, const double *f_np, const double *f_V,
                    double *x_ne, double *x_np, double *x_V, double eta, int max_cycles,
                    double *history, int *cycles, int where);

/* One backward-Euler step of length dt (eq. 7) solved by Newton-Raphson with
 * multigrid (eq. 14) until every field's rho <= tol.  On rejection (Newton cap,
 * correction limit, linear failure, non-finite) the state is unchanged and the
 * return value is MG_ENOCONV or MG_ENONFINITE.  stats may be NULL. */
int mg_step(mg_state *s, double dt, double tol, mg_stats *stats);

/* March with the Delta-t ramp of Sec. 2 from dt_start until the steady
 * residual <= tol (MG_EREJECT if max_steps is exhausted first). */
int mg_march(mg_state *s, double dt_start, double tol, mg_stats *stats);

/* Steady state by the continuation of Sec. 2 / abstract: the current state and
 * sources are injected onto the grid coarsened by two, marched there from dt1
 * to steady, prolonged bilinearly back, and marched on the full grid starting
 * with the long step dt_max, until the steady residual <= tol. */
int mg_solve_steady(mg_state *s, double tol, mg_stats *stats);

/* Steady state from an initial guess of the full-grid state (the learned-guess form, see
 * unet.h): the current state is saved, (ne, np, V) become the state (electrode rows set to
 * their Dirichlet values) and the march starts at guess_dt_start, growing by dt_growth up to
 * guess_dt_max (the paper's growing ramp, Sec. 2).  If that march fails or
 * needs more than 60 steps, the saved state is restored and mg_solve_steady's continuation
 * runs instead (*used_fallback = 1). */
int mg_solve_steady_guess(mg_state *s, const double *ne, const double *np, const double *V, int where, double tol,
                          mg_stats *stats, int *used_fallback);

/* Batched form: solve n independent discharges (the paper solves one discharge at a time,
 * Sec. 2) to their steady states (mg_solve_steady on each).
 *   workers = 0: the persistent work-list form.  Every discharge's whole steady solve (the
 *     continuation, the Delta-t march with accept / reject, the Newton iterations and the
 *     V-cycle loops, as mg_solve_steady runs them) happens in ONE launch of a persistent kernel,
 *     replayed from a captured CUDA graph.  Each discharge has a program of phases (the
 *     single-discharge path's kernels in its order); the CTAs claim work items (rounds of a
 *     phase's thread blocks, the size chosen by mg_autotune_batch) of whichever discharge has a
 *     phase open, and the CTA that completes a phase runs that discharge's march, step and
 *     Newton control on the device and opens its next phase.  Same results bit for bit as
 *     mg_solve_steady on each state (state, steps, Newton iterations, V-cycles).  Needs the
 *     point smoother, the Picard Jacobian, the coarse-cycle kernel (coarse_kernel_n > 0) at or
 *     below the continuation's first grid and a coarsest level of at most 48 unknowns;
 *     otherwise the call falls back to 16 host threads.  ms_out[k]: from the launch's start to
 *     discharge k's solve ending (device clock).  A launch in which no phase completes for 5 s
 *     ends with MG_ETIMEOUT.  n = 0 returns MG_OK at once.
 *   workers > 0: the comparison form: `workers` host threads take instances from a shared queue
 *     and run mg_solve_steady on each state's own stream (give each state a distinct stream at
 *     mg_create so that the GPU can overlap them), every linear solve a device-side CUDA-graph
 *     loop; ms_out[k]: instance k's wall time from its start to its stream being idle.
 * rc_out[k] (may be NULL) receives instance k's status.  Returns MG_OK or the first failing
 * instance's status; MG_EINVAL for workers < 0.  The states must live on the calling thread's
 * current device and must not be used by other threads during the call. */
int mg_solve_steady_batch(mg_state **states, int n, double tol, int workers, double *ms_out, int *rc_out);

/* Autotuner of the batched form's work list (mg_solve_steady_batch with workers = 0): solves
 * the n discharges to tol in one persistent launch once per candidate shape and keeps the
 * fastest in every state: the size of a work item (2, 4 or 8 rounds of 256 nodes, or of the
 * single-discharge kernel's thread blocks) and the largest level (16, 32 or 64 intervals per
 * side) from which a V-cycle's coarse part runs as one single-CTA phase (same results: only the
 * schedule changes).  *grain_out (may be NULL) receives size + 100 x level.  The states'
 * solutions, statistics and start data are restored afterwards.  MG_EINVAL when a state does
 * not qualify for the persistent form (see mg_solve_steady_batch). */
int mg_autotune_batch(mg_state **states, int n, double tol, int *grain_out);

/* Autotuner of the smoother's launch shapes: times the red-black half sweep and the fused
 * sweep of every level (FP64 and, in the mixed form, FP32) over fixed sets of thread-block /
 * tile shapes and keeps the fastest per level.  Leaves the solution state untouched (only
 * the correction work buffers are written); on each level the FP32 fused sweep is kept only
 * where it beats two half sweeps by more than 3 %, and the FP64 view always uses half sweeps
 * (their ring recompute makes fused FP64 sweeps slower inside a V-cycle).  shapes_out (may be NULL) receives 6 ints per level: FP64 half-sweep
 * (bx, by), FP64 fused flag, FP32 half-sweep (bx, by), FP32 fused flag. */
int mg_autotune(mg_state *s, int32_t *shapes_out);

/* Sets the smoother's launch on one level by hand (what mg_autotune chooses): precision 0 for
 * the FP64 view, 1 for the FP32 view (mixed form); half sweeps in blocks of bx * by threads
 * (one per node of the colour) with bx in {32, 64, 128} and bx * by <= 256; fused = 1 for one tiled launch per sweep with tile shape
 * `tile` (0: 32x2, 1: 32x4, 2: 32x8, 3: 64x2, 4: 64x4, 5: 128x2), 0 for two half sweeps.
 * Results are the same bit for bit whatever the choice.  MG_EINVAL on a bad level or shape. */
int mg_set_smoother(mg_state *s, int level, int precision, int bx, int by, int fused, int tile);

/* Pre- and post-smoothing sweeps of one level by hand, instead of the rule of the parameters
 * (nu1 / nu2, nu_coarse_n / nu_coarse1 / nu_coarse2); nu1 = nu2 = -1 restores the rule.
 * MG_EINVAL on a bad level or counts (both set or both -1, at least one sweep). */
int mg_set_level_sweeps(mg_state *s, int level, int nu1, int nu2);
int mg_num_levels(const mg_state *s);

/* Statistics accumulated since creation (or the last mg_reset_stats). */
int mg_get_stats(const mg_state *s, mg_stats *out);
void mg_reset_stats(mg_state *s);

/* Number of CUDA kernels this library has launched (all states, process-wide). */
uint64_t mg_kernel_launches(void);

/* Allocation-free residual norms.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory (code running inside another framework's memory
 * pool, real-time loops where cudaMalloc is forbidden or would synchronise the device, plug-ins
 * that may only use the buffers their host hands them).  It evaluates the same residual rows
 * and scale-free norms rho[3] as mg_residual (up to rounding: it evaluates every face directly
 * instead of through stored face coefficients), without creating a state:
 * every array argument is caller-owned DEVICE memory of (nz + 1) x (nr + 1) doubles (dense
 * rows, i fastest) and rho is host memory.  ne_old, np_old, V_old are read only when dt > 0
 * (dt <= 0: steady residual).  F_ne, F_np, F_V receive the rows when non-NULL (all three or
 * none).  The electrode rows of the inputs must hold the Dirichlet values.
 * Limits: nr, nz powers of two with 2 <= nr, nz <= 1024; at most 64 table rows; the zero-flux
 * wall only (wall_dirichlet = 1 returns MG_EINVAL); larger inputs return MG_EINVAL.  It calls no cudaMalloc, cudaFree or allocating library routine:
 * its scratch (about 232 KB: geometry, table, block partial sums, a reduction counter and the
 * results) is one file-scope device array that every GPU loading the library holds until
 * the process exits.  All calls share that array and it keeps the last call's contents, so
 * calls that overlap on the GPU race; serialise them (one stream, or synchronise between
 * calls).  The first call on a device looks up the array's device address (once per device,
 * with that device current); make that first call before any stream capture.  The call
 * synchronises `stream` (a cudaStream_t, NULL = legacy default stream) before returning. */
int mg_residual_noalloc(const mg_grid *g, const mg_params *p, const double *ne, const double *np, const double *V,
                        const double *ne_old, const double *np_old, const double *V_old, const double *S_e,
                        const double *S_p, double dt, double *F_ne, double *F_np, double *F_V, double rho[3],
                        void *stream);

#ifdef __cplusplus
}
#endif
#endif
