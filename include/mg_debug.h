/*
 * mg_debug.h - instrumentation of the GB300 multigrid solver (include/mg.h): kernel timing and
 * probes that the benchmark and the profiling cases use to attribute time to kernels and to
 * measure the FP64 rate the stencils run against.  None of these is part of the solver's
 * interface (the paper's problem statement, Sec. 2, has no counterpart); they change no result.
 */
#ifndef PAPER_0811_4446_GB300_MG_DEBUG_H
#define PAPER_0811_4446_GB300_MG_DEBUG_H

#include "mg.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Kernel timing for measurement: between mg_profile_begin and mg_profile_end every launch
 * of `kernel` on multigrid level `level` (0 = finest) is bracketed by CUDA events recorded on
 * the state's stream (up to 16384 launches).  mg_profile_end synchronises the stream and
 * returns the number of bracketed launches and their summed device time in milliseconds.
 * MG_PROF_RESTRICT brackets the fused linear-residual + restriction launch from `level`,
 * MG_PROF_LINRES the residual-norm launch of each cycle of a linear solve rooted at `level`.
 * MG_PROF_RESIDUAL brackets the face-coefficient and residual launches of a residual
 * evaluation on `level`; MG_PROF_COEF the hierarchy set-up below a Newton iteration on root
 * level `level` (injection, coarse-level coefficients and the diagonal factors of every level,
 * one launch each); MG_PROF_COARSE the launches of the coarse-cycle kernel that starts on
 * `level`; MG_PROF_COARSE_FACTOR the coarsest-level inverse below a Newton iteration on root
 * level `level`. */
enum { MG_PROF_SMOOTH = 1, MG_PROF_LINRES = 2, MG_PROF_COEF = 3, MG_PROF_RESIDUAL = 4,
       MG_PROF_RESTRICT = 5, MG_PROF_PROLONG = 6, MG_PROF_COARSE = 7, MG_PROF_COARSE_FACTOR = 8 };
int mg_profile_begin(mg_state *s, int kernel, int level);
int mg_profile_end(mg_state *s, int64_t *launches, double *total_ms);

/* Measured FP64 fused-multiply-add throughput of the current device in GFLOP/s (2 flops per
 * FMA), from a kernel of independent FMA chains on every SM; used as the ALU roofline of the
 * FP64 path.  Returns a negative value on a CUDA error. */
double mg_probe_fp64_gflops(void *stream);

/* Smoother timing as the V-cycle graphs run it: `sweeps` red-black sweeps of level `level`
 * (0 = finest, below the last level) in the precision view `precision` (0 FP64, 1 the FP32
 * view of the mixed form), issued exactly as a V-cycle issues them (the level's launch shape,
 * half or fused sweeps, programmatic dependent launch), are captured into one CUDA graph on
 * the state's stream and replayed twice; the second replay is timed with CUDA events.
 * *us_per_launch receives its device time divided by the number of launches,
 * *launches_per_sweep (may be NULL) 2 for half sweeps, 1 for fused ones.  Only the level's
 * correction buffers are written, and they are zeroed afterwards; the solution state is not
 * touched.  Synchronises the stream.  MG_EINVAL on a bad level, precision (1 needs the mixed
 * form) or sweep count (1 .. 4096); MG_ECUDA on a CUDA error. */
int mg_time_smoother(mg_state *s, int level, int precision, int sweeps, double *us_per_launch,
                     int *launches_per_sweep);

/* Launch mode of the learned-guess network (unet.h): on = 1 (the default) runs a forward pass
 * and a loss-and-gradient pass as CUDA graphs per batch size, on = 0 launch by launch, so that a
 * kernel profiler sees and attributes every launch (the results are the same). */
typedef struct mg_unet mg_unet;
int mg_unet_set_graphs(mg_unet *n, int on);

/* The network's activations after its last forward pass, for per-layer tests: which = 0 the
 * input (8 channels, bf16), 1 .. 11 the outputs of e0a, e0b, e1a, e1b, e2a, e2b, e3a, e3b, d2,
 * d1, d0 (after ReLU), 12 .. 14 the node-aligned upsampled inputs of d2, d1, d0 (from e3b, d2,
 * d1).  hwc (3 ints, may be NULL) receives the layer's grid nodes H, W and channels C; out
 * (host, may be NULL for the sizes alone) receives the bit patterns of the B x H x W x C bf16
 * values, NHWC.  Synchronises the stream.  MG_EINVAL for a bad index or B outside
 * 1 .. batch_max; MG_ECUDA on a CUDA error. */
int mg_unet_get_activation(mg_unet *n, int which, int B, uint16_t *out, int *hwc);

#ifdef __cplusplus
}
#endif
#endif
