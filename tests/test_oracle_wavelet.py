"""Pins of the oracle's Deslauriers-Dubuc derivative (Section 2.3)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle.wavelet import dd_mask, derivative_weights

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "dd_derivative_weights.txt")


def _golden():
    w, m = {}, {}
    for line in open(GOLDEN):
        t = line.split()
        if not t or t[0].startswith("#"):
            continue
        if t[0] == "mask":
            m[(int(t[1]), int(t[2]))] = Fraction(int(t[3]), int(t[4]))
        else:
            w[(int(t[0]), int(t[1]))] = Fraction(int(t[2]), int(t[3]))
    return w, m


@pytest.mark.parametrize("p", [2, 3])
def test_weights_match_closed_forms(p):
    gw, gm = _golden()
    d = derivative_weights(p)
    assert sorted(d) == [l for l in range(-(2 * p - 2), 2 * p - 1) if l != 0]
    for l in range(1, 2 * p - 1):
        ref = float(gw[(p, l)])
        assert d[l] == pytest.approx(ref, abs=1e-13)
        assert d[-l] == pytest.approx(-ref, abs=1e-13)          # odd symmetry of phi'
    h = dd_mask(p)
    for (pp, k), v in gm.items():
        if pp == p:
            assert h[k] == pytest.approx(float(v), abs=1e-15)
            assert h[-k] == pytest.approx(float(v), abs=1e-15)


@pytest.mark.parametrize("p", [2, 3])
def test_polynomial_exactness(p):
    """Section 2.3: the derivative is exact for polynomials of degree <= 2p-1.

    The odd-symmetric stencil is also exact at degree 2p (even error terms
    cancel); degree 2p+1 is the first that is not reproduced.
    """
    d = derivative_weights(p)
    dx = 0.37
    x0 = 1.3
    for q in range(0, 2 * p + 2):
        approx = sum(dl * (x0 - l * dx) ** q for l, dl in d.items()) / dx
        exact = q * x0 ** (q - 1) if q > 0 else 0.0
        if q <= 2 * p:
            assert approx == pytest.approx(exact, rel=1e-11, abs=1e-11)
        else:
            assert abs(approx - exact) > 1e-6


def _cascade(p, levels):
    """phi on the dyadic grid 2^-levels by repeated DD midpoint insertion from delta_0."""
    nodes = np.arange(-p + 1, p + 1)
    w = []
    for m in nodes:
        others = nodes[nodes != m]
        w.append(np.prod((0.5 - others) / (m - others)))
    span = 2 * p                                   # pad so boundary effects stay outside support
    vals = np.zeros(4 * span + 1)
    vals[2 * span] = 1.0
    x = np.arange(-2 * span, 2 * span + 1, dtype=float)
    for _ in range(levels):
        new = np.zeros(2 * vals.size - 1)
        new[::2] = vals
        for i in range(vals.size - 1):
            acc = 0.0
            for m, wm in zip(nodes, w):
                j = i + int(m)
                if 0 <= j < vals.size:
                    acc += wm * vals[j]
            new[2 * i + 1] = acc
        vals = new
        x = np.linspace(x[0], x[-1], vals.size)
    return x, vals


@pytest.mark.parametrize("p", [2, 3])
def test_weights_equal_derivative_of_cascade_limit(p):
    """phi'(l) from the eigen-problem equals the slope of the subdivision limit function."""
    x, phi = _cascade(p, 11)
    hh = x[1] - x[0]
    d = derivative_weights(p)
    for l in range(-(2 * p - 1), 2 * p):
        i = int(round((l - x[0]) / hh))
        slope = (-phi[i + 2] + 8 * phi[i + 1] - 8 * phi[i - 1] + phi[i - 2]) / (12 * hh)
        assert slope == pytest.approx(d.get(l, 0.0), abs=2e-4)


@pytest.mark.parametrize("p", [2, 3])
def test_fourier_symbol_and_order(p):
    """On a periodic grid D e^{ikx} = i k~ e^{ikx}, k~ dx = 2 sum_l c_l sin(l k dx), error O(dx^{2p})."""
    d = derivative_weights(p)
    errs = []
    for n in (32, 64, 128):
        dx = 2 * math.pi / n
        x = np.arange(n) * dx
        f = np.sin(3 * x)
        df = np.zeros(n)
        for l, dl in d.items():
            df += dl * np.roll(f, l)
        df /= dx
        ktil = 2 * sum(-d[l] * math.sin(l * 3 * dx) for l in d if l > 0) / dx
        assert np.allclose(df, ktil * np.cos(3 * x), atol=1e-12)
        errs.append(np.max(np.abs(df - 3 * np.cos(3 * x))))
    if p == 2:  # textbook fourth-order central-difference symbol
        dx = 2 * math.pi / 64
        assert ktil_p2(3, dx) == pytest.approx(
            2 * sum(-d[l] * math.sin(l * 3 * dx) for l in d if l > 0) / dx, rel=1e-13)
    order = math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2])
    assert min(order) > 2 * p - 0.2


def ktil_p2(k, dx):
    return (8 * math.sin(k * dx) - math.sin(2 * k * dx)) / (6 * dx)
