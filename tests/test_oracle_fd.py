"""Pins for oracle.fd: central finite-difference weights (Eq. 1 discretised, Eq. 2).

Independent checks: textbook stencils (Fornberg, Math. Comp. 51 (1988), Table 1 and
the standard 2nd-order formulas; fixture tests/golden/central_fd_weights.txt), symmetry,
and the measured convergence order on a smooth periodic function.
"""
import math
import os
from fractions import Fraction as F

import numpy as np
import pytest

from oracle import fd


GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "central_fd_weights.txt")


def _golden_weights():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.split("#", 1)[0].split()
            if line:
                rows.append((int(line[0]), int(line[1]), [F(t) for t in line[2:]]))
    return rows


@pytest.mark.parametrize("k,p,expected", _golden_weights())
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
