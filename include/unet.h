/*
 * unet.h - C ABI of the learned initial guess for the steady solver of mg.h.
 *
 * The paper (arXiv:0811.4446) reaches the steady state on the fine grid from a steady state
 * on the grid coarsened by two ("multilevel prolongation", Sec. 2).  This optional form
 * replaces that coarse-grid solve by a guess from a small U-Net (no counterpart in the paper):
 * per-node features -> (log n_e, log n_p, V) on the same node grid; the Newton-multigrid
 * march then refines the guess to the requested residual (mg_solve_steady_guess in mg.h).
 *
 * Network (fixed): 3x3 convolutions with ReLU, node grids H -> (H-1)/2+1 three times,
 *   e0a 8->32, e0b 32->32 | e1a s2 32->64, e1b 64->64 | e2a s2 64->96, e2b 96->96 |
 *   e3a s2 96->128, e3b 128->128 | d2 [up(e3b), e2b] 224->64 | d1 [up(d2), e1b] 128->32 |
 *   d0 [up(d1), e0b] 64->32 | head 1x1 32->3 (linear);  648,291 parameters.
 * "up" is node-aligned bilinear interpolation.  Activations are BF16 (NHWC), convolutions are
 * implicit GEMMs on tensor cores with FP32 accumulation; master weights, gradients and the
 * Adam moments are FP32.
 *
 * Parameter vector (FP32): for each layer in the order above its weights w[kh][kw][c_in][c_out]
 * followed by its biases b[c_out].
 * Input x: B x H x W x 8 FP32 (NHWC; channels 5..7 zero), output y: B x H x W x 3 FP32.
 * `where`: MG_HOST or MG_DEVICE (mg.h) for the caller arrays.  Calls synchronise the stream.
 * The kernels of a forward pass, and of a loss-and-gradient pass, run as a CUDA graph per batch
 * size (captured on the network's own stream at the first call with that size, replayed on the
 * caller's stream); the input copies, the Adam update and the bf16 weight copies are launched
 * around it.
 * Return values: MG_OK or a negative MG_E* code of mg.h.
 */
#ifndef PAPER_0811_4446_GB300_UNET_H
#define PAPER_0811_4446_GB300_UNET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_unet mg_unet;

int64_t mg_unet_param_count(void);

/* Network for batches of up to batch_max samples on grids of n_intervals + 1 nodes per side
 * (n_intervals a multiple of 8).  Allocates its device memory; stream = cudaStream_t. */
int mg_unet_create(int batch_max, int n_intervals, void *stream, mg_unet **out);
void mg_unet_destroy(mg_unet *n);
const char *mg_unet_last_error(const mg_unet *n);

/* Set / read the FP32 parameter vector (setting resets the optimizer). */
int mg_unet_set_params(mg_unet *n, const float *p, int where);
int mg_unet_get_params(mg_unet *n, float *p, int where);

/* Forward pass of B samples. */
int mg_unet_forward(mg_unet *n, const float *x, int B, float *y, int where);

/* Mean-squared error of the forward pass against targets t (B x H x W x 3) and its gradient
 * with respect to every parameter (read with mg_unet_get_grads); no update. */
int mg_unet_loss_grad(mg_unet *n, const float *x, const float *t, int B, double *loss, int where);
int mg_unet_get_grads(mg_unet *n, float *g, int where);

/* Tensor-core path of the convolutions: a parity and measurement reference, not a choice a
 * user makes.  The network runs on path 3 (the default), which assigns one kernel to each
 * layer shape:
 *   - the halo-load tcgen05 kernel: the forward of the stride-1 layers whose weights fit in
 *     72 KB (the 8-channel first layer included) and the stride-1 data gradients whose reversed
 *     weights fit;
 *   - the TMA-tile tcgen05 kernel: the other 3x3 forward convolutions, the other stride-1 data
 *     gradients (one launch per input part where the parts have more than 128 channels in all),
 *     and the stride-2 data gradients;
 *   - the TMA-fed tcgen05 weight gradient: every 3x3 layer;
 *   - FP32 CUDA-core kernels: the 1x1 head, forward and backward.
 * Paths 0-2 keep the earlier kernels of those layers so that the tests can compare each layer's
 * kernel with the one it replaced (same operands, another order of the sums) and the benchmark
 * can report what each replacement gained:
 *   0 = mma.sync for every convolution.
 *   1 = tcgen05.mma with the accumulator in tensor memory for the forward and data-gradient
 *       convolutions whose output width is a multiple of 16 (<= 256) and the weight gradients
 *       with 32 <= output channels <= 128, operands gathered by threads (for the weight
 *       gradient MN-major, straight from the NHWC tensors); the 1x1 head, forward and backward,
 *       on FP32 CUDA-core kernels; the rest on mma.sync.
 *   2 = as 1, except that the forward 3x3 convolutions (stride 1 or 2) whose input parts have a
 *       multiple of 32 channels take their operands by TMA tiled loads (tiles of 16 x 8 output
 *       pixels, the padding read as the loads' zero fill) in a persistent kernel.
 *   3 (default) = as 2, except that
 *       - the stride-1 forward convolutions whose weight matrix fits in 72 KB (the 8-channel
 *         first layer too) keep it resident in shared memory and load one 10 x 18-pixel halo
 *         per 32-channel chunk (8-channel plane) for all nine taps (tiles of 8 x 16 pixels);
 *       - the data gradient runs as a forward convolution of the output gradient: for stride 1
 *         with the taps reversed, on the halo kernel where the reversed weights fit, else on the
 *         tile kernel; for stride 2 on the tile kernel over the output gradient's own grid, once
 *         per parity class of the input pixels (the 1, 2, 2 or 4 taps that reach it);
 *       - the weight gradient of the 3x3 layers takes both operands by TMA tiled loads (segments
 *         of 64 or 128 output pixels, one load per tap and 32-channel slice, or 8-channel slice
 *         for the first layer).
 *       Their sums round in another order.
 * Any other value returns MG_EINVAL.  A tcgen05 kernel whose bounded wait expires makes the next
 * call return MG_ETIMEOUT. */
int mg_unet_set_tensor_path(mg_unet *n, int path);

/* One training step: loss and gradients as above, then an Adam update (beta1 0.9,
 * beta2 0.999, eps 1e-8) with learning rate lr. */
int mg_unet_train_step(mg_unet *n, const float *x, const float *t, int B, float lr, double *loss, int where);

#ifdef __cplusplus
}
#endif
#endif
