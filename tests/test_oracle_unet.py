"""Pins for the CPU oracle of the learned-initial-guess network (oracle/unet.py).

* autograd gradients = central finite differences (float64, random directions);
* the 3x3 convolution with the [kh][kw][c_in][c_out] weight layout, zero padding and
  stride 2 = a brute-force sum over the stencil;
* node-aligned upsampling reproduces bilinear functions exactly;
* the first Adam step moves each parameter by lr * g / (|g| + eps).
"""
import numpy as np
import pytest
import torch

from oracle import unet


def test_param_count_matches_layer_table():
    n = 0
    for _, k, _, ci, co, _ in unet.LAYERS:
        n += k * k * ci * co + co
    assert unet.param_count() == n == 648291


@pytest.mark.parametrize("stride", [1, 2])
def test_conv_matches_brute_force(stride):
    g = torch.Generator().manual_seed(1)
    x = torch.randn(2, 3, 9, 9, generator=g, dtype=torch.float64)
    w = torch.randn(3, 3, 3, 4, generator=g, dtype=torch.float64)
    b = torch.randn(4, generator=g, dtype=torch.float64)
    y = unet.conv(x, w, b, stride)
    Ho = (9 + 2 - 3) // stride + 1
    ref = np.zeros((2, 4, Ho, Ho))
    xn, wn = x.numpy(), w.numpy()
    for n in range(2):
        for co in range(4):
            for yo in range(Ho):
                for xo in range(Ho):
                    acc = b[co].item()
                    for kh in range(3):
                        for kw in range(3):
                            yi, xi = yo * stride + kh - 1, xo * stride + kw - 1
                            if 0 <= yi < 9 and 0 <= xi < 9:
                                acc += sum(xn[n, ci, yi, xi] * wn[kh, kw, ci, co] for ci in range(3))
                    ref[n, co, yo, xo] = acc
    assert np.allclose(y.numpy(), ref, rtol=1e-13, atol=1e-13)


def test_upsample_exact_for_bilinear():
    h = 5
    I, J = np.meshgrid(np.arange(h), np.arange(h))
    f = lambda a, b: 1.0 + 2.0 * a - 0.5 * b + 0.25 * a * b
    x = torch.tensor(f(I, J), dtype=torch.float64)[None, None]
    up = unet.upsample_nodes(x)[0, 0].numpy()
    I2, J2 = np.meshgrid(np.arange(2 * h - 1) / 2.0, np.arange(2 * h - 1) / 2.0)
    assert np.allclose(up, f(I2, J2), rtol=1e-14, atol=1e-14)


def test_autograd_matches_finite_differences():
    torch.manual_seed(0)
    p = unet.init_params(3)
    for k in p:
        if k.endswith(".b"):
            p[k] = 0.1 * torch.randn_like(p[k])
    x = torch.randn(2, 8, 17, 17, dtype=torch.float64)
    t = torch.randn(2, 3, 17, 17, dtype=torch.float64)
    loss, grads = unet.loss_and_grads(p, x, t)
    flat = unet.flatten(p)
    gflat = unet.flatten(grads)
    for trial in range(3):
        d = torch.randn_like(flat)
        d /= d.norm()                      # unit direction: no ReLU kink is crossed
        eps = 1e-5
        lp = float(unet.mse_loss(unet.forward(unet.unflatten(flat + eps * d), x), t))
        lm = float(unet.mse_loss(unet.forward(unet.unflatten(flat - eps * d), x), t))
        fd = (lp - lm) / (2 * eps)
        an = float(gflat @ d)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-6), (trial, fd, an)


def test_first_adam_step():
    p = {"a": torch.tensor([0.5, -1.0, 2.0], dtype=torch.float64)}
    gr = {"a": torch.tensor([0.3, -2.0, 1e-3], dtype=torch.float64)}
    m = {"a": torch.zeros(3, dtype=torch.float64)}
    v = {"a": torch.zeros(3, dtype=torch.float64)}
    lr = 1e-2
    new, _, _ = unet.adam_step(dict(p), gr, m, v, 1, lr)
    expect = p["a"] - lr * gr["a"] / (gr["a"].abs() + 1e-8)
    assert torch.allclose(new["a"], expect, rtol=1e-12, atol=1e-15)
