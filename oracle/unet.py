"""Plain CPU oracle of the learned initial guess (a small U-Net on the node grid).

Test infrastructure only.  The paper has no learned component; this network is the
"learned initial guess" form of the solver: it maps per-node problem features (cathode
voltage, pressure factor, source map, r and z) to a guess of the steady state
(log n_e, log n_p, V) that replaces the coarse-grid part of the continuation (Sec. 2).
Plain PyTorch CPU ops in float64; backward by autograd (pinned in the tests by central
finite differences).

Architecture (node grids 257 -> 129 -> 65 -> 33 for a 257 x 257 input; any 8k + 1 size):
  e0a 3x3 s1  8->32   e0b 3x3 s1 32->32                 (skip0)
  e1a 3x3 s2 32->64   e1b 3x3 s1 64->64                 (skip1)
  e2a 3x3 s2 64->96   e2b 3x3 s1 96->96                 (skip2)
  e3a 3x3 s2 96->128  e3b 3x3 s1 128->128
  d2: up(e3b) ++ skip2 (224) 3x3 -> 64
  d1: up(d2)  ++ skip1 (128) 3x3 -> 32
  d0: up(d1)  ++ skip0 (64)  3x3 -> 32
  head 1x1 32 -> 3 (no activation)
All 3x3 convolutions have zero padding 1 and are followed by ReLU.  "up" is node-aligned
bilinear interpolation to the grid of twice the intervals (coarse node k = fine node 2k).
Channel counts: the 5 input features are padded with zeros to 8 channels.
Weights are stored as [kh][kw][c_in][c_out] (K x N with K = (kh, kw, c_in)), biases [c_out].
"""
from __future__ import annotations

from typing import Dict, List, Tuple

import torch
import torch.nn.functional as Fn

# (name, kernel size, stride, c_in, c_out, relu)
LAYERS: List[Tuple[str, int, int, int, int, bool]] = [
    ("e0a", 3, 1, 8, 32, True), ("e0b", 3, 1, 32, 32, True),
    ("e1a", 3, 2, 32, 64, True), ("e1b", 3, 1, 64, 64, True),
    ("e2a", 3, 2, 64, 96, True), ("e2b", 3, 1, 96, 96, True),
    ("e3a", 3, 2, 96, 128, True), ("e3b", 3, 1, 128, 128, True),
    ("d2", 3, 1, 224, 64, True), ("d1", 3, 1, 128, 32, True), ("d0", 3, 1, 64, 32, True),
    ("head", 1, 1, 32, 3, False),
]
IN_CH, OUT_CH = 8, 3


def param_count() -> int:
    return sum(k * k * ci * co + co for _, k, _, ci, co, _ in LAYERS)


def init_params(seed: int = 0, dtype=torch.float64) -> Dict[str, torch.Tensor]:
    """He-normal weights, zero biases (seeded)."""
    g = torch.Generator().manual_seed(seed)
    p = {}
    for name, k, _, ci, co, _ in LAYERS:
        std = (2.0 / (k * k * ci)) ** 0.5
        p[name + ".w"] = torch.randn(k, k, ci, co, generator=g, dtype=torch.float64).to(dtype) * std
        p[name + ".b"] = torch.zeros(co, dtype=dtype)
    return p


def flatten(params: Dict[str, torch.Tensor]) -> torch.Tensor:
    """All parameters in layer order (w then b of each layer) as one vector."""
    return torch.cat([torch.cat([params[n + ".w"].reshape(-1), params[n + ".b"]]) for n, *_ in LAYERS])


def unflatten(v: torch.Tensor, dtype=torch.float64) -> Dict[str, torch.Tensor]:
    p, o = {}, 0
    for name, k, _, ci, co, _ in LAYERS:
        nw = k * k * ci * co
        p[name + ".w"] = v[o:o + nw].reshape(k, k, ci, co).to(dtype)
        o += nw
        p[name + ".b"] = v[o:o + co].to(dtype)
        o += co
    return p


def conv(x: torch.Tensor, w: torch.Tensor, b: torch.Tensor, stride: int) -> torch.Tensor:
    """x: (B, C_in, H, W); w: [kh][kw][c_in][c_out]; zero padding (k - 1) / 2."""
    k = w.shape[0]
    wt = w.permute(3, 2, 0, 1)           # (c_out, c_in, kh, kw): the layout conv2d expects
    return Fn.conv2d(x, wt, b, stride=stride, padding=(k - 1) // 2)


def upsample_nodes(x: torch.Tensor) -> torch.Tensor:
    """Node-aligned bilinear interpolation (B, C, h, w) -> (B, C, 2h - 1, 2w - 1)."""
    B, C, h, w = x.shape
    out = x.new_zeros(B, C, 2 * h - 1, 2 * w - 1)
    out[:, :, ::2, ::2] = x
    out[:, :, ::2, 1::2] = 0.5 * (x[:, :, :, :-1] + x[:, :, :, 1:])
    out[:, :, 1::2, :] = 0.5 * (out[:, :, 0:-1:2, :] + out[:, :, 2::2, :])
    return out


def forward(params: Dict[str, torch.Tensor], x: torch.Tensor, keep: bool = False):
    """x: (B, 8, H, W) -> (B, 3, H, W).  keep=True also returns every layer's output."""
    acts = {}

    def layer(name, inp):
        _, k, s, ci, co, relu = next(l for l in LAYERS if l[0] == name)
        y = conv(inp, params[name + ".w"], params[name + ".b"], s)
        y = torch.relu(y) if relu else y
        acts[name] = y
        return y

    s0 = layer("e0b", layer("e0a", x))
    s1 = layer("e1b", layer("e1a", s0))
    s2 = layer("e2b", layer("e2a", s1))
    b3 = layer("e3b", layer("e3a", s2))
    d2 = layer("d2", torch.cat([upsample_nodes(b3), s2], dim=1))
    d1 = layer("d1", torch.cat([upsample_nodes(d2), s1], dim=1))
    d0 = layer("d0", torch.cat([upsample_nodes(d1), s0], dim=1))
    y = layer("head", d0)
    return (y, acts) if keep else y


def mse_loss(y: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
    return ((y - target) ** 2).mean()


def loss_and_grads(params: Dict[str, torch.Tensor], x: torch.Tensor, target: torch.Tensor):
    """(loss, dict of gradients) by autograd in the parameters' dtype."""
    p = {k: v.detach().clone().requires_grad_(True) for k, v in params.items()}
    loss = mse_loss(forward(p, x), target)
    loss.backward()
    return float(loss.detach()), {k: v.grad.detach() for k, v in p.items()}


def adam_step(params, grads, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) in place; m, v are the moment dicts."""
    for k in params:
        m[k] = beta1 * m[k] + (1 - beta1) * grads[k]
        v[k] = beta2 * v[k] + (1 - beta2) * grads[k] ** 2
        mh = m[k] / (1 - beta1 ** step)
        vh = v[k] / (1 - beta2 ** step)
        params[k] = params[k] - lr * mh / (vh.sqrt() + eps)
    return params, m, v
