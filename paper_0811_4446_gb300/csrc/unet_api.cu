// Host side of include/unet.h: the learned-initial-guess network (a U-Net on the node grid)
// on BF16 tensor-core convolution kernels (unet_kernels.cu).  The network maps per-node problem
// features (cathode voltage, pressure factor, source map, r, z) to a guess of the steady state
// (log n_e, log n_p, V) that replaces the coarse-grid part of the continuation of Sec. 2 of
// arXiv:0811.4446; the paper itself has no learned component.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/mg.h"
#include "../../include/mg_debug.h"
#include "../../include/unet.h"
#include "unet_impl.cuh"

using namespace unk;

namespace {

struct LayerDef {
  int ks, stride, ci, co, relu;
};
// e0a e0b e1a e1b e2a e2b e3a e3b d2 d1 d0 head (same order as the parameter vector)
constexpr int NL = 12;
constexpr LayerDef kL[NL] = {{3, 1, 8, 32, 1},   {3, 1, 32, 32, 1},   {3, 2, 32, 64, 1},  {3, 1, 64, 64, 1},
                             {3, 2, 64, 96, 1},  {3, 1, 96, 96, 1},   {3, 2, 96, 128, 1}, {3, 1, 128, 128, 1},
                             {3, 1, 224, 64, 1}, {3, 1, 128, 32, 1}, {3, 1, 64, 32, 1},  {1, 1, 32, 3, 0}};
enum { E0A, E0B, E1A, E1B, E2A, E2B, E3A, E3B, D2, D1, D0, HEAD };

int pad8(int c) { return (c + 7) & ~7; }

struct Act {
  __nv_bfloat16 *a = nullptr;  // activation, NHWC bf16
  float *g = nullptr;          // gradient, NHWC FP32
  bool gw = false;             // g holds a contribution of the current backward pass
  int H = 0, W = 0, C = 0;
  size_t elems(int B) const { return (size_t)B * H * W * C; }
};

}  // namespace

struct mg_unet {
  int Bmax = 0, H = 0;
  cudaStream_t st = nullptr;
  size_t nparam = 0, woff[NL], boff[NL];
  float *master = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16 *wf[NL], *wd[NL], *wdf[NL];
  float *dwpad = nullptr;
  Act x, e0a, e0b, e1a, e1b, e2a, e2b, e3a, e3b, u3, d2, u2, d1, u1, d0;
  float *out = nullptr, *dout = nullptr, *tgt = nullptr, *xin = nullptr;
  __nv_bfloat16 *dpre = nullptr, *dpre2 = nullptr;  // a layer's bf16 output gradient, by layer parity
  __nv_bfloat16 *dpre_head = nullptr;  // the head's output gradient when d0's output stage folds it in
  double *loss_d = nullptr, *loss_h = nullptr;
  int *tc_err = nullptr;   // set by a tcgen05 kernel whose bounded wait expired
  int use_tc = 3;          // 1: tcgen05 where the layer shape allows it; 2: TMA-fed where it can; 3: halo loads too
  ConvMaps maps[NL];       // tensor maps of the TMA-fed forward convolutions, built on first use
  const void *map_key[NL][4] = {};  // inputs, weights and the kind of map (2: tile boxes, 3: halo boxes)
  ConvMaps wmaps[NL];      // tensor maps of the TMA-fed weight gradients, built on first use
  const void *wmap_key[NL][3] = {};  // their inputs and dY
  ConvMaps dmaps[NL];      // tensor maps of the TMA-fed data gradients, built on first use
  ConvMaps dmaps2[NL];     // ... of the second input part where the parts run as two launches
  const void *dmap_key[NL][3] = {};  // their dY, weights and the kind of map (2: tile, 3: halo, 4: parity,
                                     // 5: tile per input part)
  int step = 0;
  void *block = nullptr;
  std::string err;
  // The kernels of a forward pass, and of forward + loss + backward, as CUDA graphs per batch
  // size for the current tensor path (captured on a private stream, launched on the caller's)
  cudaStream_t cap = nullptr;
  std::vector<cudaGraphExec_t> gfwd, gtrain;
  cudaStream_t side = nullptr;            // a layer's weight gradient beside the later layers' work
  cudaEvent_t ev_fork = nullptr, ev_join[3] = {nullptr, nullptr, nullptr};  // per dY buffer
  int graphs = 1;          // 0: launch by launch (mg_unet_set_graphs, for kernel profilers)
};

namespace {

int fail(mg_unet *n, int code, const char *fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (n) n->err = buf;
  return code;
}

#define UK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail(n, MG_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

size_t param_count() {
  size_t p = 0;
  for (const auto &l : kL) p += (size_t)l.ks * l.ks * l.ci * l.co + l.co;
  return p;
}

// one carve of the device block (sizes only when base == nullptr)
struct Carve {
  char *base;
  size_t off;
  template <typename T>
  T *take(size_t count) {
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += (count * sizeof(T) + 255) & ~size_t(255);
    return p;
  }
};

void layout(mg_unet *n, Carve &c) {
  const int B = n->Bmax, H0 = n->H, H1 = (H0 - 1) / 2 + 1, H2 = (H1 - 1) / 2 + 1, H3 = (H2 - 1) / 2 + 1;
  n->nparam = param_count();
  size_t o = 0;
  size_t maxw = 0;
  for (int l = 0; l < NL; ++l) {
    n->woff[l] = o;
    o += (size_t)kL[l].ks * kL[l].ks * kL[l].ci * kL[l].co;
    n->boff[l] = o;
    o += kL[l].co;
    maxw = std::max(maxw, (size_t)kL[l].ks * kL[l].ks * kL[l].ci * pad8(kL[l].co));
  }
  n->master = c.take<float>(n->nparam);
  n->grad = c.take<float>(n->nparam);
  n->m = c.take<float>(n->nparam);
  n->v = c.take<float>(n->nparam);
  for (int l = 0; l < NL; ++l) {
    const size_t e = (size_t)kL[l].ks * kL[l].ks * kL[l].ci * pad8(kL[l].co);
    n->wf[l] = c.take<__nv_bfloat16>(e);
    n->wd[l] = c.take<__nv_bfloat16>(e);
    n->wdf[l] = c.take<__nv_bfloat16>(e);
  }
  n->dwpad = c.take<float>(maxw);
  auto act = [&](Act &t, int Hh, int C) {
    t.H = t.W = Hh;
    t.C = C;
    t.a = c.take<__nv_bfloat16>(t.elems(B));
    t.g = c.take<float>(t.elems(B));
  };
  act(n->x, H0, 8);
  act(n->e0a, H0, 32); act(n->e0b, H0, 32);
  act(n->e1a, H1, 64); act(n->e1b, H1, 64);
  act(n->e2a, H2, 96); act(n->e2b, H2, 96);
  act(n->e3a, H3, 128); act(n->e3b, H3, 128);
  act(n->u3, H2, 128); act(n->d2, H2, 64);
  act(n->u2, H1, 64); act(n->d1, H1, 32);
  act(n->u1, H0, 32); act(n->d0, H0, 32);
  const size_t P0 = (size_t)B * H0 * H0;
  n->out = c.take<float>(P0 * 8);
  n->dout = c.take<float>(P0 * 8);
  n->tgt = c.take<float>(P0 * 3);
  n->xin = c.take<float>(P0 * 8);
  n->dpre = c.take<__nv_bfloat16>(P0 * 32);
  n->dpre2 = c.take<__nv_bfloat16>(P0 * 32);
  n->dpre_head = c.take<__nv_bfloat16>(P0 * 8);
  n->loss_d = c.take<double>(1);
  n->tc_err = c.take<int>(4);
}

ConvArgs conv_args(const mg_unet *n, int l, int B, const Act &in1, const Act *in2) {
  ConvArgs a;
  std::memset(&a, 0, sizeof(a));
  const LayerDef &L = kL[l];
  a.Bn = B;
  a.Hin = in1.H; a.Win = in1.W;
  a.ks = L.ks; a.stride = L.stride; a.pad = (L.ks - 1) / 2;
  a.Hout = (a.Hin + 2 * a.pad - a.ks) / a.stride + 1;
  a.Wout = (a.Win + 2 * a.pad - a.ks) / a.stride + 1;
  a.C1 = in1.C; a.C2 = in2 ? in2->C : 0;
  a.Cout = pad8(L.co);
  a.Pout = B * a.Hout * a.Wout;
  a.Kf = a.ks * a.ks * (a.C1 + a.C2);
  a.x1 = in1.a; a.x2 = in2 ? in2->a : nullptr;
  a.bias = n->master + n->boff[l];
  a.Nreal = L.co;
  a.relu = L.relu;
  return a;
}

int conv_fwd(mg_unet *n, int l, int B, const Act &in1, const Act *in2, Act *out, float *out32) {
  ConvArgs a = conv_args(n, l, B, in1, in2);
  a.M = a.Pout; a.N = a.Cout; a.K = a.Kf;
  a.w = n->wf[l];
  a.y = out ? out->a : nullptr;
  a.y32 = out32;
  if (n->use_tc && conv1x1_f32_supported(a)) {
    UK(launch_conv1x1_f32(a, n->st));
  } else if (n->use_tc == 3 && conv_halo_supported(a, MODE_FWD)) {
    const void *key[4] = {a.x1, a.x2, a.w, reinterpret_cast<const void *>(3)};
    if (std::memcmp(key, n->map_key[l], sizeof(key)) != 0) {
      if (int rc = make_halo_maps(a, n->Bmax, &n->maps[l]))
        return fail(n, MG_ECUDA, "halo tensor maps of layer %d: encode step %d failed", l, rc);
      std::memcpy(n->map_key[l], key, sizeof(key));
    }
    UK(launch_conv_halo(a, n->maps[l], n->tc_err, n->st));
  } else if (n->use_tc >= 2 && conv_tma_supported(a, MODE_FWD)) {
    const void *key[4] = {a.x1, a.x2, a.w, reinterpret_cast<const void *>(2)};
    if (std::memcmp(key, n->map_key[l], sizeof(key)) != 0) {
      if (int rc = make_conv_maps(a, n->Bmax, &n->maps[l]))
        return fail(n, MG_ECUDA, "tensor maps of layer %d: encode step %d failed", l, rc);
      std::memcpy(n->map_key[l], key, sizeof(key));
    }
    UK(launch_conv_tma(a, n->maps[l], n->tc_err, n->st));
  } else if (n->use_tc && conv_tc_supported(a, MODE_FWD)) {
    UK(launch_conv_tc(a, MODE_FWD, n->tc_err, n->st));
  } else {
    UK(launch_conv(a, MODE_FWD, 1, n->st));
  }
  return MG_OK;
}

// Backward of layer l given the FP32 gradient of its output (out.g, or dout32 for the head):
// ReLU mask, weight and bias gradients, and (if want_dx) the data gradient added into the
// inputs' gradients.
// The first data-gradient contribution to an activation's gradient overwrites it (no zeroing
// pass, no read), later ones add; returns the data-gradient kernels' dacc flag in *dacc.
int dx_mode(mg_unet *n, int B, Act &in1, Act *in2, int *dacc) {
  const bool w1 = in1.gw, w2 = in2 ? in2->gw : w1;
  if (w1 != w2) {
    Act &z = w1 ? *in2 : in1;
    UK(cudaMemsetAsync(z.g, 0, z.elems(B) * sizeof(float), n->st));
  }
  *dacc = (w1 || w2) ? 1 : 0;
  in1.gw = true;
  if (in2) in2->gw = true;
  return MG_OK;
}

// The weight gradient of layer l (GEMM (kh, kw, ci) x cop over the output pixels) on stream st:
// added straight into the (zeroed) gradient vector where no output channel is padded, else into
// the padded buffer and copied over
int wgrad_part(mg_unet *n, int l, const ConvArgs &a, const __nv_bfloat16 *dpre, cudaStream_t st) {
  const int cop = a.Cout;
  ConvArgs w = a;
  w.M = a.Kf; w.N = cop; w.K = a.Pout;
  w.dy = dpre;
  const bool padded = cop != kL[l].co;
  w.dw = padded ? n->dwpad : n->grad + n->woff[l];
  if (padded) UK(cudaMemsetAsync(n->dwpad, 0, (size_t)a.Kf * cop * sizeof(float), st));
  if (n->use_tc && conv1x1_bwd_supported(a)) {
    UK(launch_conv1x1_wgrad(a, dpre, n->dwpad, st));
  } else if (n->use_tc == 3 && wgrad_tma_supported(w)) {
    const void *key[3] = {w.x1, w.x2, w.dy};
    if (std::memcmp(key, n->wmap_key[l], sizeof(key)) != 0) {
      if (int rc = make_wgrad_maps(w, n->Bmax, &n->wmaps[l]))
        return fail(n, MG_ECUDA, "weight-gradient tensor maps of layer %d: encode step %d failed", l, rc);
      std::memcpy(n->wmap_key[l], key, sizeof(key));
    }
    UK(launch_wgrad_tma(w, n->wmaps[l], n->tc_err, st));
  } else if (n->use_tc && wgrad_tc_supported(w)) {
    UK(launch_wgrad_tc(w, n->tc_err, st));
  } else {
    const int tiles = ((w.M + 63) / 64) * ((w.N + 63) / 64);
    const int splits = std::max(1, std::min((w.K + 255) / 256, 2 * 152 * 2 / std::max(1, tiles)));
    UK(launch_conv(w, MODE_WGRAD, splits, st));
  }
  if (padded) UK(launch_unpad_grad(n->dwpad, n->grad + n->woff[l], (size_t)a.Kf, kL[l].co, cop, st));
  return MG_OK;
}

// The data gradient of layer l into its inputs' gradients, on the network's stream
int dgrad_part(mg_unet *n, int l, int B, const ConvArgs &a, Act &in1, Act *in2, const __nv_bfloat16 *dpre,
               bool want_dx) {
  const int cop = a.Cout;
  int dacc = 1;
  if (want_dx)
    if (int rc = dx_mode(n, B, in1, in2, &dacc)) return rc;
  if (want_dx && n->use_tc == 3 && a.ks == 3 && a.stride == 2) {
    // stride 2: the tile kernel on dY's own grid, once per output parity class (the taps that
    // reach that class), with the data-gradient weights wd
    ConvArgs f;
    std::memset(&f, 0, sizeof(f));
    f.Bn = B;
    f.Hin = f.Hout = a.Hout;
    f.Win = f.Wout = a.Wout;
    f.ks = 3; f.stride = 1; f.pad = 1;
    f.C1 = cop; f.C2 = 0;
    f.x1 = dpre;
    f.N = f.Cout = f.Nreal = a.C1 + a.C2;
    f.M = B * a.Hout * a.Wout; f.K = 9 * cop; f.Kf = f.K; f.Pout = f.M;
    f.w = n->wd[l];
    f.dx1 = in1.g; f.dx2 = in2 ? in2->g : nullptr; f.dsplit = a.C1; f.dacc = dacc;
    if (conv_tma_supported(f, MODE_FWD)) {
      const void *key[3] = {f.x1, f.w, reinterpret_cast<const void *>(4)};
      if (std::memcmp(key, n->dmap_key[l], sizeof(key)) != 0) {
        if (int rc = make_conv_maps(f, n->Bmax, &n->dmaps[l]))
          return fail(n, MG_ECUDA, "data-gradient tensor maps of layer %d: encode step %d failed", l, rc);
        std::memcpy(n->dmap_key[l], key, sizeof(key));
      }
      UK(launch_conv_tma_parity(f, n->dmaps[l], a.Hin, a.Win, n->tc_err, n->st));
      return MG_OK;
    }
  }
  if (want_dx && n->use_tc == 3 && a.ks == 3 && a.stride == 1) {
    // stride 1: dX = dY convolved with the reversed taps (wdf), a forward convolution on the
    // input grid: on the halo kernel where the reversed weights fit in 72 KB, else on the TMA tile
    // kernel where the input parts have at most 128 channels in all
    ConvArgs f;
    std::memset(&f, 0, sizeof(f));
    f.Bn = B;
    f.Hin = f.Hout = a.Hin;
    f.Win = f.Wout = a.Win;
    f.ks = 3; f.stride = 1; f.pad = 1;
    f.C1 = cop; f.C2 = 0;
    f.x1 = dpre;
    f.N = f.Cout = f.Nreal = a.C1 + a.C2;
    f.M = B * a.Hin * a.Win; f.K = 9 * cop; f.Kf = f.K; f.Pout = f.M;
    f.w = n->wdf[l];
    f.dx1 = in1.g; f.dx2 = in2 ? in2->g : nullptr; f.dsplit = a.C1; f.dacc = dacc;
    const bool halo = conv_halo_supported(f, MODE_FWD);
    if (halo || conv_tma_supported(f, MODE_FWD)) {
      const void *key[3] = {f.x1, f.w, reinterpret_cast<const void *>(halo ? 3 : 2)};
      if (std::memcmp(key, n->dmap_key[l], sizeof(key)) != 0) {
        if (int rc = halo ? make_halo_maps(f, n->Bmax, &n->dmaps[l]) : make_conv_maps(f, n->Bmax, &n->dmaps[l]))
          return fail(n, MG_ECUDA, "data-gradient tensor maps of layer %d: encode step %d failed", l, rc);
        std::memcpy(n->dmap_key[l], key, sizeof(key));
      }
      if (halo) UK(launch_conv_halo(f, n->dmaps[l], n->tc_err, n->st));
      else UK(launch_conv_tma(f, n->dmaps[l], n->tc_err, n->st));
      return MG_OK;
    }
    // wider than one tile kernel's 128 outputs (d2): one launch per input part, each with its
    // rows of the reversed weights
    ConvArgs f1 = f, f2 = f;
    f1.N = f1.Cout = f1.Nreal = a.C1; f1.dsplit = a.C1; f1.dx2 = nullptr;
    f2.N = f2.Cout = f2.Nreal = a.C2; f2.dsplit = a.C2; f2.dx1 = f.dx2; f2.dx2 = nullptr;
    f2.w = f.w + (size_t)a.C1 * f.K;
    if (a.C2 > 0 && conv_tma_supported(f1, MODE_FWD) && conv_tma_supported(f2, MODE_FWD)) {
      const void *key[3] = {f.x1, f.w, reinterpret_cast<const void *>(5)};
      if (std::memcmp(key, n->dmap_key[l], sizeof(key)) != 0) {
        if (int rc = make_conv_maps(f1, n->Bmax, &n->dmaps[l]))
          return fail(n, MG_ECUDA, "data-gradient tensor maps of layer %d: encode step %d failed", l, rc);
        if (int rc = make_conv_maps(f2, n->Bmax, &n->dmaps2[l]))
          return fail(n, MG_ECUDA, "data-gradient tensor maps of layer %d: encode step %d failed", l, rc);
        std::memcpy(n->dmap_key[l], key, sizeof(key));
      }
      UK(launch_conv_tma(f1, n->dmaps[l], n->tc_err, n->st));
      UK(launch_conv_tma(f2, n->dmaps2[l], n->tc_err, n->st));
      return MG_OK;
    }
  }
  if (want_dx) {
    ConvArgs d = a;
    d.M = B * a.Hin * a.Win; d.N = a.C1 + a.C2; d.K = a.ks * a.ks * cop;
    d.w = n->wd[l];
    d.dy = dpre;
    d.dx1 = in1.g;
    d.dx2 = in2 ? in2->g : nullptr;
    d.dacc = dacc;
    if (n->use_tc && conv_tc_supported(d, MODE_DGRAD)) UK(launch_conv_tc(d, MODE_DGRAD, n->tc_err, n->st));
    else UK(launch_conv(d, MODE_DGRAD, 1, n->st));
  }
  return MG_OK;
}

// dpre_buf (may be null: dpre) receives the layer's bf16 output gradient; head_dy (may be null)
// makes the layer's output stage the fused head data gradient + ReLU + bias pass
int conv_bwd(mg_unet *n, int l, int B, Act &in1, Act *in2, const Act *out, const float *dout32, bool want_dx,
             __nv_bfloat16 *dpre_buf = nullptr, const __nv_bfloat16 *head_dy = nullptr) {
  // the layer's dY buffer: its own (the head's) or one of two by layer parity, which the weight
  // gradient of the layer two steps back (on the side stream) must have finished reading
  const int jb = dpre_buf ? 2 : (l & 1);
  __nv_bfloat16 *const dpre = dpre_buf ? dpre_buf : ((l & 1) ? n->dpre2 : n->dpre);
  if (n->side) UK(cudaStreamWaitEvent(n->st, n->ev_join[jb], 0));
  ConvArgs a = conv_args(n, l, B, in1, in2);
  const size_t P = (size_t)a.Pout;
  const int cop = a.Cout;
  if (head_dy)
    UK(launch_head_relu_bias_bwd(head_dy, n->wd[HEAD], out->a, dpre, n->grad + n->boff[l], (int)P, cop, kL[l].co,
                                 n->st));
  else
    UK(launch_relu_bias_bwd(out ? out->g : dout32, out ? out->a : nullptr, dpre, n->grad + n->boff[l], (int)P, cop,
                            kL[l].co, out ? kL[l].relu : 0, n->st));
  // the weight and the data gradient are independent (one reads the input and dY, the other dY
  // and the weights): the weight gradient runs on the side stream beside the data gradient and
  // the later layers' work, until the layer two steps on reuses this dY buffer
  if (n->side) {
    UK(cudaEventRecord(n->ev_fork, n->st));
    UK(cudaStreamWaitEvent(n->side, n->ev_fork, 0));
    if (int rc = wgrad_part(n, l, a, dpre, n->side)) return rc;
    UK(cudaEventRecord(n->ev_join[jb], n->side));
    return dgrad_part(n, l, B, a, in1, in2, dpre, want_dx);
  }
  if (int rc = wgrad_part(n, l, a, dpre, n->st)) return rc;
  return dgrad_part(n, l, B, a, in1, in2, dpre, want_dx);
}

int refresh_weights(mg_unet *n) {
  static_assert(NL <= kMaxWeightCopies, "weight-copy table");
  WeightCopies c;
  std::memset(&c, 0, sizeof(c));
  c.n = NL;
  for (int l = 0; l < NL; ++l)
    c.l[l] = {n->master + n->woff[l], n->wf[l], n->wd[l], n->wdf[l], kL[l].ks, kL[l].ci, kL[l].co, pad8(kL[l].co)};
  UK(launch_weight_copies(c, n->st));
  return MG_OK;
}

int forward(mg_unet *n, int B) {
  int rc;
  const Act &x = n->x;
  if ((rc = conv_fwd(n, E0A, B, x, nullptr, &n->e0a, nullptr))) return rc;
  if ((rc = conv_fwd(n, E0B, B, n->e0a, nullptr, &n->e0b, nullptr))) return rc;
  if ((rc = conv_fwd(n, E1A, B, n->e0b, nullptr, &n->e1a, nullptr))) return rc;
  if ((rc = conv_fwd(n, E1B, B, n->e1a, nullptr, &n->e1b, nullptr))) return rc;
  if ((rc = conv_fwd(n, E2A, B, n->e1b, nullptr, &n->e2a, nullptr))) return rc;
  if ((rc = conv_fwd(n, E2B, B, n->e2a, nullptr, &n->e2b, nullptr))) return rc;
  if ((rc = conv_fwd(n, E3A, B, n->e2b, nullptr, &n->e3a, nullptr))) return rc;
  if ((rc = conv_fwd(n, E3B, B, n->e3a, nullptr, &n->e3b, nullptr))) return rc;
  UK(launch_upsample(n->e3b.a, n->u3.a, B, n->e3b.H, n->e3b.W, n->e3b.C, n->st));
  if ((rc = conv_fwd(n, D2, B, n->u3, &n->e2b, &n->d2, nullptr))) return rc;
  UK(launch_upsample(n->d2.a, n->u2.a, B, n->d2.H, n->d2.W, n->d2.C, n->st));
  if ((rc = conv_fwd(n, D1, B, n->u2, &n->e1b, &n->d1, nullptr))) return rc;
  UK(launch_upsample(n->d1.a, n->u1.a, B, n->d1.H, n->d1.W, n->d1.C, n->st));
  if ((rc = conv_fwd(n, D0, B, n->u1, &n->e0b, &n->d0, nullptr))) return rc;
  return conv_fwd(n, HEAD, B, n->d0, nullptr, nullptr, n->out);
}

int backward(mg_unet *n, int B) {
  int rc;
  Act *all[] = {&n->x, &n->e0a, &n->e0b, &n->e1a, &n->e1b, &n->e2a, &n->e2b, &n->e3a,
                &n->e3b, &n->u3, &n->d2, &n->u2, &n->d1, &n->u1, &n->d0};
  for (Act *t : all) t->gw = false;
  // the dY buffers' events start out complete in this stream's order (and inside a capture)
  if (n->side)
    for (auto &e : n->ev_join) UK(cudaEventRecord(e, n->st));
  UK(cudaMemsetAsync(n->grad, 0, n->nparam * sizeof(float), n->st));
  // with the head's backward on the CUDA cores its data gradient is folded into d0's output
  // stage (never stored): the head's bf16 output gradient goes to its own buffer for that
  const ConvArgs ha = conv_args(n, HEAD, B, n->d0, nullptr);
  const bool fold = n->use_tc && conv1x1_bwd_supported(ha) && kL[D0].relu && kL[D0].co == n->d0.C;
  if ((rc = conv_bwd(n, HEAD, B, n->d0, nullptr, nullptr, n->dout, !fold, fold ? n->dpre_head : nullptr))) return rc;
  if ((rc = conv_bwd(n, D0, B, n->u1, &n->e0b, &n->d0, nullptr, true, nullptr, fold ? n->dpre_head : nullptr)))
    return rc;
  UK(launch_upsample_bwd(n->u1.g, n->d1.g, B, n->d1.H, n->d1.W, n->d1.C, n->st));
  n->d1.gw = true;
  if ((rc = conv_bwd(n, D1, B, n->u2, &n->e1b, &n->d1, nullptr, true))) return rc;
  UK(launch_upsample_bwd(n->u2.g, n->d2.g, B, n->d2.H, n->d2.W, n->d2.C, n->st));
  n->d2.gw = true;
  if ((rc = conv_bwd(n, D2, B, n->u3, &n->e2b, &n->d2, nullptr, true))) return rc;
  UK(launch_upsample_bwd(n->u3.g, n->e3b.g, B, n->e3b.H, n->e3b.W, n->e3b.C, n->st));
  n->e3b.gw = true;
  if ((rc = conv_bwd(n, E3B, B, n->e3a, nullptr, &n->e3b, nullptr, true))) return rc;
  if ((rc = conv_bwd(n, E3A, B, n->e2b, nullptr, &n->e3a, nullptr, true))) return rc;
  if ((rc = conv_bwd(n, E2B, B, n->e2a, nullptr, &n->e2b, nullptr, true))) return rc;
  if ((rc = conv_bwd(n, E2A, B, n->e1b, nullptr, &n->e2a, nullptr, true))) return rc;
  if ((rc = conv_bwd(n, E1B, B, n->e1a, nullptr, &n->e1b, nullptr, true))) return rc;
  if ((rc = conv_bwd(n, E1A, B, n->e0b, nullptr, &n->e1a, nullptr, true))) return rc;
  if ((rc = conv_bwd(n, E0B, B, n->e0a, nullptr, &n->e0b, nullptr, true))) return rc;
  if ((rc = conv_bwd(n, E0A, B, n->x, nullptr, &n->e0a, nullptr, false))) return rc;
  // every weight gradient is in before the caller reads the gradients or Adam runs
  if (n->side)
    for (auto &e : n->ev_join) UK(cudaStreamWaitEvent(n->st, e, 0));
  return MG_OK;
}

cudaMemcpyKind kin(int where) { return where == MG_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }
cudaMemcpyKind kout(int where) { return where == MG_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }

// a tcgen05 kernel that gave up on a bounded wait leaves the flag set
int check_tc(mg_unet *n) {
  int h = 0;
  UK(cudaMemcpy(&h, n->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    cudaMemset(n->tc_err, 0, sizeof(int));
    return fail(n, MG_ETIMEOUT, "tensor-core convolution: bounded wait expired");
  }
  return MG_OK;
}

int load_input(mg_unet *n, const float *x, int B, int where) {
  const size_t e = (size_t)B * n->H * n->H * 8;
  UK(cudaMemcpyAsync(n->xin, x, e * sizeof(float), kin(where), n->st));
  return MG_OK;
}

// the device work of a forward pass from the FP32 input in xin
int forward_body(mg_unet *n, int B) {
  UK(launch_f32_to_bf16(n->xin, n->x.a, (size_t)B * n->H * n->H * 8, n->st));
  return forward(n, B);
}

// ... and of the loss against the targets in tgt and the backward pass
int train_body(mg_unet *n, int B) {
  int rc = forward_body(n, B);
  if (rc) return rc;
  const size_t P = (size_t)B * n->H * n->H;
  UK(cudaMemsetAsync(n->loss_d, 0, sizeof(double), n->st));
  UK(launch_mse(n->out, n->tgt, n->dout, P, 8, 3, n->loss_d, n->st));
  return backward(n, B);
}

void drop_graphs(mg_unet *n) {
  for (auto *v : {&n->gfwd, &n->gtrain})
    for (auto &g : *v)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
}

// Runs body's kernels for batch size B as a CUDA graph: captured on the private stream the first
// time (the host-side choices of every launch, tensor maps included, are fixed for a batch size
// and tensor path), then launched on the caller's stream.  If capturing fails the body runs
// launch by launch.
int run_graph(mg_unet *n, std::vector<cudaGraphExec_t> &cache, int B, int (*body)(mg_unet *, int)) {
  if (!n->graphs) return body(n, B);
  if (!cache[B] && n->cap) {
    cudaStream_t user = n->st;
    n->st = n->cap;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(n->cap, cudaStreamCaptureModeThreadLocal);
    int rc = e == cudaSuccess ? body(n, B) : MG_ECUDA;
    if (e == cudaSuccess) e = cudaStreamEndCapture(n->cap, &g);
    n->st = user;
    if (rc == MG_OK && e == cudaSuccess && g) e = cudaGraphInstantiate(&cache[B], g, 0);
    if (g) cudaGraphDestroy(g);
    if (rc != MG_OK || e != cudaSuccess) {
      cache[B] = nullptr;
      cudaGetLastError();
      return body(n, B);
    }
  }
  if (!cache[B]) return body(n, B);
  UK(cudaGraphLaunch(cache[B], n->st));
  return MG_OK;
}

int loss_grad(mg_unet *n, const float *x, const float *t, int B, double *loss, int where) {
  if (!n || !x || !t || B < 1 || B > n->Bmax) return MG_EINVAL;
  int rc;
  const size_t P = (size_t)B * n->H * n->H;
  if ((rc = load_input(n, x, B, where))) return rc;
  UK(cudaMemcpyAsync(n->tgt, t, P * 3 * sizeof(float), kin(where), n->st));
  if ((rc = run_graph(n, n->gtrain, B, train_body))) return rc;
  UK(cudaMemcpyAsync(n->loss_h, n->loss_d, sizeof(double), cudaMemcpyDeviceToHost, n->st));
  UK(cudaStreamSynchronize(n->st));
  if (loss) *loss = *n->loss_h;
  return check_tc(n);
}

}  // namespace

extern "C" {

int64_t mg_unet_param_count(void) { return (int64_t)param_count(); }

int mg_unet_create(int batch_max, int n_intervals, void *stream, mg_unet **out) {
  if (!out) return MG_EINVAL;
  *out = nullptr;
  if (batch_max < 1 || n_intervals < 8 || n_intervals % 8) return MG_EINVAL;
  mg_unet *n = new (std::nothrow) mg_unet();
  if (!n) return MG_ENOMEM;
  n->Bmax = batch_max;
  n->H = n_intervals + 1;
  n->st = (cudaStream_t)stream;
  Carve sz{nullptr, 0};
  layout(n, sz);
  if (cudaMalloc(&n->block, sz.off) != cudaSuccess) { delete n; return MG_ENOMEM; }
  if (cudaMallocHost(&n->loss_h, sizeof(double)) != cudaSuccess) { cudaFree(n->block); delete n; return MG_ECUDA; }
  Carve c{(char *)n->block, 0};
  layout(n, c);
  if (cudaMemsetAsync(n->block, 0, sz.off, n->st) != cudaSuccess || cudaStreamSynchronize(n->st) != cudaSuccess ||
      cudaStreamCreateWithFlags(&n->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&n->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&n->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&n->ev_join[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&n->ev_join[1], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&n->ev_join[2], cudaEventDisableTiming) != cudaSuccess) {
    mg_unet_destroy(n);
    return MG_ECUDA;
  }
  n->gfwd.assign(batch_max + 1, nullptr);
  n->gtrain.assign(batch_max + 1, nullptr);
  *out = n;
  return MG_OK;
}

void mg_unet_destroy(mg_unet *n) {
  if (!n) return;
  cudaStreamSynchronize(n->st);  // the caller's stream (null: the legacy default stream)
  drop_graphs(n);
  if (n->side) cudaStreamSynchronize(n->side);
  if (n->ev_fork) cudaEventDestroy(n->ev_fork);
  for (auto &e : n->ev_join)
    if (e) cudaEventDestroy(e);
  if (n->side) cudaStreamDestroy(n->side);
  if (n->cap) cudaStreamDestroy(n->cap);
  if (n->block) cudaFree(n->block);
  if (n->loss_h) cudaFreeHost(n->loss_h);
  delete n;
}

const char *mg_unet_last_error(const mg_unet *n) { return n ? n->err.c_str() : "null network"; }

int mg_unet_set_params(mg_unet *n, const float *p, int where) {
  if (!n || !p) return MG_EINVAL;
  UK(cudaMemcpyAsync(n->master, p, n->nparam * sizeof(float), kin(where), n->st));
  UK(cudaMemsetAsync(n->m, 0, n->nparam * sizeof(float), n->st));
  UK(cudaMemsetAsync(n->v, 0, n->nparam * sizeof(float), n->st));
  n->step = 0;
  int rc = refresh_weights(n);
  if (rc) return rc;
  UK(cudaStreamSynchronize(n->st));
  return MG_OK;
}

int mg_unet_get_params(mg_unet *n, float *p, int where) {
  if (!n || !p) return MG_EINVAL;
  UK(cudaMemcpyAsync(p, n->master, n->nparam * sizeof(float), kout(where), n->st));
  UK(cudaStreamSynchronize(n->st));
  return MG_OK;
}

int mg_unet_get_grads(mg_unet *n, float *g, int where) {
  if (!n || !g) return MG_EINVAL;
  UK(cudaMemcpyAsync(g, n->grad, n->nparam * sizeof(float), kout(where), n->st));
  UK(cudaStreamSynchronize(n->st));
  return MG_OK;
}

int mg_unet_forward(mg_unet *n, const float *x, int B, float *y, int where) {
  if (!n || !x || !y || B < 1 || B > n->Bmax) return MG_EINVAL;
  int rc;
  if ((rc = load_input(n, x, B, where)) || (rc = run_graph(n, n->gfwd, B, forward_body))) return rc;
  // out is [P][8]; copy the 3 real channels with a pitched copy
  const size_t P = (size_t)B * n->H * n->H;
  UK(cudaMemcpy2DAsync(y, 3 * sizeof(float), n->out, 8 * sizeof(float), 3 * sizeof(float), P, kout(where), n->st));
  UK(cudaStreamSynchronize(n->st));
  return check_tc(n);
}

int mg_unet_set_graphs(mg_unet *n, int on) {
  if (!n || (on != 0 && on != 1)) return MG_EINVAL;
  n->graphs = on;
  return MG_OK;
}

int mg_unet_get_activation(mg_unet *n, int which, int B, uint16_t *out, int *hwc) {
  if (!n || which < 0 || which > 14 || B < 1 || B > n->Bmax) return MG_EINVAL;
  const Act *all[] = {&n->x,   &n->e0a, &n->e0b, &n->e1a, &n->e1b, &n->e2a, &n->e2b, &n->e3a,
                      &n->e3b, &n->d2,  &n->d1,  &n->d0,  &n->u3,  &n->u2,  &n->u1};
  const Act &t = *all[which];
  if (hwc) { hwc[0] = t.H; hwc[1] = t.W; hwc[2] = t.C; }
  if (!out) return MG_OK;
  UK(cudaMemcpyAsync(out, t.a, t.elems(B) * sizeof(__nv_bfloat16), cudaMemcpyDeviceToHost, n->st));
  UK(cudaStreamSynchronize(n->st));
  return MG_OK;
}

int mg_unet_set_tensor_path(mg_unet *n, int path) {
  if (!n || path < 0 || path > 3) return MG_EINVAL;
  if (path != n->use_tc) {
    if (cudaStreamSynchronize(n->st) != cudaSuccess) return fail(n, MG_ECUDA, "set_tensor_path: stream sync");
    drop_graphs(n);
  }
  n->use_tc = path;
  return MG_OK;
}

int mg_unet_loss_grad(mg_unet *n, const float *x, const float *t, int B, double *loss, int where) {
  return loss_grad(n, x, t, B, loss, where);
}

int mg_unet_train_step(mg_unet *n, const float *x, const float *t, int B, float lr, double *loss, int where) {
  int rc = loss_grad(n, x, t, B, loss, where);
  if (rc) return rc;
  n->step++;
  UK(launch_adam(n->master, n->grad, n->m, n->v, n->nparam, lr, n->step, n->st));
  return refresh_weights(n);
}

}  // extern "C"
