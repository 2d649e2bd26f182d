"""Pins for the Bernoulli functions F, G of the Scharfetter-Gummel flux (Sec. 2, after eq. 11).

Reference values come from a 50-digit ``decimal`` evaluation of the printed
definitions F(x) = x/(e^x - 1), G(x) = x e^x/(e^x - 1), independent of the
oracle's series / expm1 split.
"""
from decimal import Decimal, getcontext

import numpy as np
import pytest

from oracle import bernoulli as bn

getcontext().prec = 60

XS = [-700.0, -60.0, -5.0, -1.0, -0.10000001, -0.1, -0.0999999, -0.03, -1e-2, -1e-5, -1e-12,
      1e-12, 1e-5, 1e-2, 0.03, 0.0999999, 0.1, 0.10000001, 0.5, 1.0, 2.0, 5.0, 30.0, 60.0, 700.0]


def _F_dec(x: float) -> Decimal:
    X = Decimal(x)
    return X / (X.exp() - 1)


def _dF_dec(x: float) -> Decimal:
    X = Decimal(x)
    e = X.exp()
    return (e - 1 - X * e) / (e - 1) ** 2


@pytest.mark.parametrize("x", XS)
def test_F_matches_50_digit_definition(x):
    ref = float(_F_dec(x))
    got = float(bn.F(np.array([x]))[0])
    if ref == 0.0:
        assert got == 0.0 or abs(got) < 1e-300
    else:
        assert abs(got - ref) <= 4e-16 * abs(ref), (x, got, ref)


@pytest.mark.parametrize("x", XS)
def test_G_matches_50_digit_definition(x):
    X = Decimal(x)
    ref = float(X * X.exp() / (X.exp() - 1))
    got = float(bn.G(np.array([x]))[0])
    if ref == 0.0:
        assert abs(got) < 1e-300
    else:
        assert abs(got - ref) <= 4e-16 * abs(ref), (x, got, ref)


@pytest.mark.parametrize("x", XS)
def test_dF_matches_50_digit_derivative(x):
    ref = float(_dF_dec(x))
    got = float(bn.dF(np.array([x]))[0])
    # the closed form loses up to ~1.5 digits just above the series cut
    assert abs(got - ref) <= 5e-14 * max(abs(ref), 1e-300) or abs(got - ref) < 1e-300, (x, got, ref)


def test_identities():
    x = np.concatenate([np.linspace(-40, 40, 2001), np.logspace(-14, 2, 200), -np.logspace(-14, 2, 200)])
    F, G = bn.F(x), bn.G(x)
    # G - F = x, F(-x) = G(x)
    assert np.allclose(G - F, x, rtol=1e-14, atol=1e-14)
    assert np.array_equal(bn.F(-x), G)
    assert np.all(F > 0) and np.all(G > 0)
    # F' and G' differ by one: G = F + x
    assert np.allclose(bn.dG(x) - bn.dF(x), 1.0, rtol=0, atol=1e-13)


def test_values_at_zero():
    assert bn.F(np.array([0.0]))[0] == 1.0
    assert bn.G(np.array([0.0]))[0] == 1.0
    assert bn.dF(np.array([0.0]))[0] == -0.5
    assert bn.dG(np.array([0.0]))[0] == 0.5


def test_continuous_across_series_cut():
    c = bn.SERIES_CUT
    for x0 in (c, -c):
        a = bn.F(np.array([np.nextafter(x0, 0.0)]))[0]
        b = bn.F(np.array([x0]))[0]
        assert abs(a - b) <= 4e-16 * abs(b)
