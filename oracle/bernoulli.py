"""Bernoulli function of the Scharfetter-Gummel flux (Sec. 2, definitions after eq. 11).

The paper defines F(x) = x / (exp(x) - 1) and G(x) = x exp(x) / (exp(x) - 1).
Both are the Bernoulli generating function B(x) = x / (e^x - 1):
F(x) = B(x) and G(x) = B(-x) = B(x) + x.

Evaluation (FP64):
* |x| < 0.1: the Taylor series of B with the Bernoulli numbers
  B_1 = -1/2, B_2 = 1/6, B_4 = -1/30, B_6 = 1/42, B_8 = -1/30, B_10 = 5/66, B_12 = -691/2730
  (B(x) = sum_n B_n x^n / n!); the first omitted term is below 1e-21 there.
* otherwise: B(x) = x / expm1(x) for x < 0, and B(x) = x e^{-x} / (-expm1(-x)) for
  x > 0, which never overflows.
Derivative B'(x) = (e^x - 1 - x e^x) / (e^x - 1)^2, with the same split.
Pinned in tests against a 50-digit ``decimal`` evaluation and the identities
G - F = x, F(-x) = G(x), F(0) = 1, B'(0) = -1/2.
"""
from __future__ import annotations

import numpy as np

SERIES_CUT = 0.1

# B_n / n! for n = 0, 1, 2, 4, 6, 8, 10, 12 (odd n > 1 vanish)
_C = {0: 1.0, 1: -0.5, 2: 1.0 / 12.0, 4: -1.0 / 720.0, 6: 1.0 / 30240.0,
      8: -1.0 / 1209600.0, 10: 1.0 / 47900160.0, 12: -691.0 / 1307674368000.0}


def _series_B(x):
    x2 = x * x
    even = _C[0] + x2 * (_C[2] + x2 * (_C[4] + x2 * (_C[6] + x2 * (_C[8] + x2 * (_C[10] + x2 * _C[12])))))
    return even + _C[1] * x


def _series_dB(x):
    # d/dx of the series: -1/2 + sum_{k>=1} 2k c_{2k} x^{2k-1}
    x2 = x * x
    odd = x * (2 * _C[2] + x2 * (4 * _C[4] + x2 * (6 * _C[6] + x2 * (8 * _C[8] + x2 * (10 * _C[10] + x2 * 12 * _C[12])))))
    return _C[1] + odd


def B(x):
    """B(x) = x / (exp(x) - 1), elementwise, FP64."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    small = np.abs(x) < SERIES_CUT
    neg = (~small) & (x < 0)
    pos = (~small) & (x > 0)
    out[small] = _series_B(x[small])
    xn = x[neg]
    out[neg] = xn / np.expm1(xn)
    xp = x[pos]
    out[pos] = xp * np.exp(-xp) / (-np.expm1(-xp))
    return out


def dB(x):
    """B'(x) = (e^x - 1 - x e^x) / (e^x - 1)^2, elementwise, FP64."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    small = np.abs(x) < SERIES_CUT
    neg = (~small) & (x < 0)
    pos = (~small) & (x > 0)
    out[small] = _series_dB(x[small])
    xn = x[neg]
    em = np.expm1(xn)
    out[neg] = (em - xn * np.exp(xn)) / (em * em)
    xp = x[pos]
    t = np.exp(-xp)
    emn = -np.expm1(-xp)          # 1 - e^{-x}
    # multiply numerator and denominator of B' by e^{-2x}
    out[pos] = t * (emn - xp) / (emn * emn)
    return out


def F(x):
    """F(x) = x / (e^x - 1) as printed after eq. 11."""
    return B(x)


def G(x):
    """G(x) = x e^x / (e^x - 1) as printed after eq. 11; equals B(-x)."""
    return B(-np.asarray(x, dtype=np.float64))


def dF(x):
    return dB(x)


def dG(x):
    return -dB(-np.asarray(x, dtype=np.float64))
