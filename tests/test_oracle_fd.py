"""Pins for oracle.fd: central finite-difference weights (Eq. 1 discretised, Eq. 2).

Independent checks: textbook stencils (Fornberg, Math. Comp. 51 (1988), Table 1 and
the standard 2nd-order formulas), symmetry, and the measured convergence order on a
smooth periodic function.
"""
import math
from fractions import Fraction as F

import numpy as np
import pytest

from oracle import fd


@pytest.mark.parametrize("k,p,expected", [
    (1, 2, [F(-1, 2), F(0), F(1, 2)]),
    (2, 2, [F(1), F(-2), F(1)]),
    (1, 4, [F(1, 12), F(-2, 3), F(0), F(2, 3), F(-1, 12)]),
    (2, 4, [F(-1, 12), F(4, 3), F(-5, 2), F(4, 3), F(-1, 12)]),
    (1, 6, [F(-1, 60), F(3, 20), F(-3, 4), F(0), F(3, 4), F(-3, 20), F(1, 60)]),
    (2, 6, [F(1, 90), F(-3, 20), F(3, 2), F(-49, 18), F(3, 2), F(-3, 20), F(1, 90)]),
    (1, 8, [F(1, 280), F(-4, 105), F(1, 5), F(-4, 5), F(0), F(4, 5), F(-1, 5), F(4, 105), F(-1, 280)]),
    (2, 8, [F(-1, 560), F(8, 315), F(-1, 5), F(8, 5), F(-205, 72), F(8, 5), F(-1, 5), F(8, 315), F(-1, 560)]),
    (3, 2, [F(-1, 2), F(1), F(0), F(-1), F(1, 2)]),
    (4, 2, [F(1), F(-4), F(6), F(-4), F(1)]),
    (4, 4, [F(-1, 6), F(2), F(-13, 2), F(28, 3), F(-13, 2), F(2), F(-1, 6)]),
])
def test_textbook_weights(k, p, expected):
    assert fd.central_weights_exact(k, p) == expected


@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("p", [2, 4, 6, 8])
def test_symmetry(k, p):
    w = fd.central_weights_exact(k, p)
    sign = 1 if k % 2 == 0 else -1
    assert all(w[j] == sign * w[-1 - j] for j in range(len(w)))
    assert sum(w) == 0  # constants have zero derivative


@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("p", [2, 4, 6, 8])
def test_convergence_order(k, p):
    """Error of d^k sin(x) on periodic grids falls like h^p."""
    errs = []
    for n in (16, 32):
        h = 2 * math.pi / n
        x = np.arange(n) * h
        u = np.sin(x)
        w = fd.central_weights(k, p)
        r = (len(w) - 1) // 2
        d = sum(w[j + r] * np.roll(u, -j) for j in range(-r, r + 1)) / h ** k
        exact = [np.cos(x), -np.sin(x), -np.cos(x), np.sin(x)][k - 1]
        errs.append(np.abs(d - exact).max())
    order = math.log2(errs[0] / errs[1])
    assert abs(order - p) < 0.3, (k, p, errs, order)
