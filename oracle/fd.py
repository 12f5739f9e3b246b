"""Central finite-difference weights for the k-th derivative terms of Eq. 1.

Eq. 1 writes the operator as a sum of alpha_ki * d^k u / dx_i^k; Eq. 2 is its
discretisation.  The paper leaves the discretisation method open; this oracle uses
central differences of even accuracy order p on the half-width

    r = floor((k - 1) / 2) + p / 2,

so that 2r + 1 points carry exactly p-th order accuracy for both even and odd k.

The weights w_j (j = -r..r) satisfy the Taylor moment conditions

    sum_j w_j j^q / q! = [q == k]      for q = 0..2r,

which this module solves exactly in rational arithmetic (Gauss-Jordan over Fractions),
so d^k u/dx^k ~= h^-k sum_j w_j u(x + j h).
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial
from typing import List


def half_width(k: int, p: int) -> int:
    if k < 1 or p < 2 or p % 2:
        raise ValueError("need derivative order k >= 1 and even accuracy order p >= 2")
    return (k - 1) // 2 + p // 2


def central_weights_exact(k: int, p: int) -> List[Fraction]:
    """Exact weights w_{-r..r} of the central difference for d^k/dx^k, accuracy p."""
    r = half_width(k, p)
    npts = 2 * r + 1
    offsets = list(range(-r, r + 1))
    # rows q = 0..2r: sum_j w_j j^q / q! = [q == k]
    mat = [[Fraction(j) ** q / factorial(q) for j in offsets] + [Fraction(int(q == k))]
           for q in range(npts)]
    # Gauss-Jordan elimination, exact
    for col in range(npts):
        piv = next(rw for rw in range(col, npts) if mat[rw][col] != 0)
        mat[col], mat[piv] = mat[piv], mat[col]
        pv = mat[col][col]
        mat[col] = [v / pv for v in mat[col]]
        for rw in range(npts):
            if rw != col and mat[rw][col] != 0:
                f = mat[rw][col]
                mat[rw] = [a - f * b for a, b in zip(mat[rw], mat[col])]
    return [mat[i][npts] for i in range(npts)]


def central_weights(k: int, p: int) -> List[float]:
    return [float(w) for w in central_weights_exact(k, p)]
