"""Learned initial guess: binding of include/unet.h plus the feature / target transforms,
training-set generation and the guess-then-refine steady solve.

All network arithmetic (convolutions, their gradients, Adam) runs in libmg.so's CUDA kernels;
this module converts arrays and sequences calls.  Features of one discharge, per node:
  0: V_cathode / -400 V      1: pressure factor - 1      2: S / 1e20 m^-3 s^-1
  3: r / R                   4: z / d                    5-7: zero
Targets: (log10(max(n, 1e8 m^-3)) - 14) / 2 for n_e and n_p, and V / |V_cathode|.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

from . import mg

N_FLOOR = 1e8
_c = ctypes
_vp, _i, _f, _d = _c.c_void_p, _c.c_int, _c.c_float, _c.c_double

SIGNATURES = {
    "mg_unet_param_count": (_c.c_int64, []),
    "mg_unet_create": (_i, [_i, _i, _vp, _c.POINTER(_vp)]),
    "mg_unet_destroy": (None, [_vp]),
    "mg_unet_last_error": (_c.c_char_p, [_vp]),
    "mg_unet_set_params": (_i, [_vp, _vp, _i]),
    "mg_unet_get_params": (_i, [_vp, _vp, _i]),
    "mg_unet_forward": (_i, [_vp, _vp, _i, _vp, _i]),
    "mg_unet_loss_grad": (_i, [_vp, _vp, _vp, _i, _c.POINTER(_d), _i]),
    "mg_unet_get_grads": (_i, [_vp, _vp, _i]),
    "mg_unet_train_step": (_i, [_vp, _vp, _vp, _i, _f, _c.POINTER(_d), _i]),
    "mg_unet_set_tensor_path": (_i, [_vp, _i]),
    "mg_unet_set_graphs": (_i, [_vp, _i]),
    "mg_unet_get_activation": (_i, [_vp, _i, _i, _vp, _c.POINTER(_i)]),
}

WEIGHTS_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights")


def _lib():
    lib = mg.load()
    if not getattr(lib, "_unet_bound", False):
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        lib._unet_bound = True
    return lib


def param_count() -> int:
    return int(_lib().mg_unet_param_count())


def _ptr32(a):
    import torch
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float32 and a.flags.c_contiguous
        return a.ctypes.data, mg.MG_HOST
    assert isinstance(a, torch.Tensor) and a.dtype == torch.float32 and a.is_contiguous()
    return a.data_ptr(), (mg.MG_DEVICE if a.is_cuda else mg.MG_HOST)


class UNet:
    def __init__(self, batch_max: int, n_intervals: int, stream=None):
        import torch
        self.lib = _lib()
        self.B, self.n = int(batch_max), int(n_intervals)
        self.H = self.n + 1
        st = stream if stream is not None else torch.cuda.current_stream()
        h = _vp()
        rc = self.lib.mg_unet_create(self.B, self.n, _vp(st.cuda_stream), _c.byref(h))
        if rc != mg.MG_OK:
            raise mg.MGError(rc, "mg_unet_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.mg_unet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != mg.MG_OK:
            raise mg.MGError(rc, self.lib.mg_unet_last_error(self.h).decode())

    def set_tensor_path(self, path: int):
        """1: tcgen05 / TMEM convolutions where the shape allows, 0: mma.sync everywhere,
        2: as 1 with TMA-fed operands for the 3x3 forward convolutions (stride 1 or 2)
        whose input parts have a multiple of 32 channels, 3 (default): as 2 with one halo load
        per 32-channel chunk for all nine taps where the weights fit in shared memory."""
        self._check(self.lib.mg_unet_set_tensor_path(self.h, int(path)))

    def set_graphs(self, on: bool):
        """Launch mode (mg_unet_set_graphs in include/mg_debug.h): CUDA graphs (default) or
        launch by launch, for kernel profilers."""
        self._check(self.lib.mg_unet_set_graphs(self.h, int(bool(on))))

    def activation(self, which: int, B: int) -> np.ndarray:
        """A layer's bf16 activations after the last forward pass (mg_unet_get_activation in
        include/mg_debug.h), as float32 (B, H, W, C): 0 the input, 1 .. 11 the outputs of e0a ..
        d0, 12 .. 14 the upsampled inputs of d2, d1, d0."""
        hwc = (_i * 3)()
        self._check(self.lib.mg_unet_get_activation(self.h, int(which), int(B), None, hwc))
        bits = np.empty((B, hwc[0], hwc[1], hwc[2]), np.uint16)
        self._check(self.lib.mg_unet_get_activation(self.h, int(which), int(B), bits.ctypes.data, hwc))
        return (bits.astype(np.uint32) << 16).view(np.float32)

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32) if isinstance(p, np.ndarray) else p
        ptr, w = _ptr32(p)
        self._check(self.lib.mg_unet_set_params(self.h, ptr, w))

    def get_params(self) -> np.ndarray:
        out = np.empty(param_count(), dtype=np.float32)
        self._check(self.lib.mg_unet_get_params(self.h, out.ctypes.data, mg.MG_HOST))
        return out

    def forward(self, x, out=None):
        """x: (B, H, W, 8) float32 -> (B, H, W, 3) float32 (same memory space as x)."""
        import torch
        B = x.shape[0]
        if out is None:
            out = (np.empty((B, self.H, self.H, 3), np.float32) if isinstance(x, np.ndarray)
                   else torch.empty((B, self.H, self.H, 3), dtype=torch.float32, device=x.device))
        px, w = _ptr32(x)
        py, _ = _ptr32(out)
        self._check(self.lib.mg_unet_forward(self.h, px, B, py, w))
        return out

    def loss_grad(self, x, t):
        loss = _d(0.0)
        px, w = _ptr32(x)
        pt, _ = _ptr32(t)
        self._check(self.lib.mg_unet_loss_grad(self.h, px, pt, x.shape[0], _c.byref(loss), w))
        g = np.empty(param_count(), dtype=np.float32)
        self._check(self.lib.mg_unet_get_grads(self.h, g.ctypes.data, mg.MG_HOST))
        return loss.value, g

    def train_step(self, x, t, lr: float) -> float:
        loss = _d(0.0)
        px, w = _ptr32(x)
        pt, _ = _ptr32(t)
        self._check(self.lib.mg_unet_train_step(self.h, px, pt, x.shape[0], float(lr), _c.byref(loss), w))
        return loss.value


# ------------------------------------------------------------------ transforms
def features(d) -> np.ndarray:
    """(H, W, 8) float32 features of a workloads.Discharge."""
    H, W = d.shape
    x = np.zeros((H, W, 8), np.float32)
    rr, zz = np.meshgrid(d.r, d.z)
    x[..., 0] = d.V_cathode / -400.0
    x[..., 1] = d.pressure_factor - 1.0
    x[..., 2] = d.S_e / 1e20
    x[..., 3] = rr / d.R
    x[..., 4] = zz / d.d
    return x


def targets(ne, np_, V, V_cathode) -> np.ndarray:
    t = np.empty(ne.shape + (3,), np.float32)
    t[..., 0] = (np.log10(np.maximum(ne, N_FLOOR)) - 14.0) / 2.0
    t[..., 1] = (np.log10(np.maximum(np_, N_FLOOR)) - 14.0) / 2.0
    t[..., 2] = V / abs(V_cathode)
    return t


def state_from_output(y: np.ndarray, V_cathode: float):
    """Inverse of targets(): (n_e, n_p, V) float64 node arrays from one (H, W, 3) output."""
    y = np.asarray(y, dtype=np.float64)
    ne = 10.0 ** (2.0 * y[..., 0] + 14.0)
    np_ = 10.0 ** (2.0 * y[..., 1] + 14.0)
    V = y[..., 2] * abs(V_cathode)
    return [np.ascontiguousarray(a) for a in (ne, np_, V)]


def guess_discharge(seed: int, n: int = 256):
    """One instance of the learned-guess family: the batch ranges of cathode voltage and
    pressure factor, its own Gaussian source, constant transport / pressure factor."""
    import workloads as W
    prm = W.unet_sample_params(seed)
    return W.make_discharge(n, seed=seed, V_cathode=prm["V_cathode"], pressure_factor=prm["pressure_factor"])


def generate(seeds: Sequence[int], n: int = 256, tol: float = 1e-8, workers: int = 16, precision=mg.MG_MIXED,
             chunk: int = 64):
    """Steady states of the seeded instances (batched solves): (X (N,H,W,8), T (N,H,W,3)) float32."""
    import torch
    X, T = [], []
    for c0 in range(0, len(seeds), chunk):
        ds = [guess_discharge(s, n) for s in seeds[c0:c0 + chunk]]
        solvers = [mg.from_discharge(d, precision=precision, stream=torch.cuda.Stream()) for d in ds]
        rc, _, rcs = mg.solve_steady_batch(solvers, tol, workers=workers)
        for d, s, r in zip(ds, solvers, rcs):
            if r != mg.MG_OK:
                continue
            ne, np_, V = s.get_state()
            X.append(features(d))
            T.append(targets(ne, np_, V, d.V_cathode))
        for s in solvers:
            s.close()
    return np.stack(X), np.stack(T)


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights, zero biases, in the parameter-vector order of unet.h."""
    rng = np.random.default_rng(seed)
    layers = [(3, 8, 32), (3, 32, 32), (3, 32, 64), (3, 64, 64), (3, 64, 96), (3, 96, 96), (3, 96, 128),
              (3, 128, 128), (3, 224, 64), (3, 128, 32), (3, 64, 32), (1, 32, 3)]
    out = []
    for k, ci, co in layers:
        out.append(rng.standard_normal(k * k * ci * co) * np.sqrt(2.0 / (k * k * ci)))
        out.append(np.zeros(co))
    return np.concatenate(out).astype(np.float32)


def train(net: UNet, X, T, epochs: int, batch: int, lr: float = 1e-3, seed: int = 0, log=None) -> List[float]:
    """Adam training on device tensors X (N,H,W,8), T (N,H,W,3); cosine learning-rate decay."""
    import math
    import torch
    N = X.shape[0]
    rng = np.random.default_rng(seed)
    steps = epochs * max(1, N // batch)
    hist, k = [], 0
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(N)).to(X.device)
        tot = 0.0
        nb = max(1, N // batch)
        for b in range(nb):
            idx = perm[b * batch:(b + 1) * batch]
            x = X.index_select(0, idx).contiguous()
            t = T.index_select(0, idx).contiguous()
            cur = lr * 0.5 * (1.0 + math.cos(math.pi * k / max(1, steps)))
            tot += net.train_step(x, t, cur)
            k += 1
        hist.append(tot / nb)
        if log:
            log(ep, hist[-1])
    return hist


def load_weights(name: str = "unet_guess_257.f32") -> Optional[np.ndarray]:
    path = os.path.join(WEIGHTS_DIR, name)
    if not os.path.exists(path):
        return None
    return np.fromfile(path, dtype=np.float32)
