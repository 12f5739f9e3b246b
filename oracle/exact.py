"""The fixed result of one implicit-Euler step: u^{n+1} = A^{-1} u^n (Eq. 4).

GMRES run to a tolerance converges to this unique vector, so it is written out here by
its plain definition, twice:

* ``solve_dense``   LU with partial pivoting of the assembled A (tiny grids);
* ``solve_fourier`` for periodic constant-coefficient stencils A is (block-)circulant:
                    every Fourier mode is multiplied by 1 / (1 - dt lambda(theta)).
"""
from __future__ import annotations

import numpy as np

from .operator import Operator


def solve_dense(op: Operator, u_n: np.ndarray, dt: float) -> np.ndarray:
    return np.linalg.solve(op.dense_A(dt), np.asarray(u_n, dtype=np.float64))


def solve_fourier(op: Operator, u_n: np.ndarray, dt: float) -> np.ndarray:
    grid = np.asarray(u_n, dtype=np.float64).reshape(tuple(reversed(op.shape)))
    amp = 1.0 / (1.0 - dt * op.symbol())
    return np.real(np.fft.ifftn(np.fft.fftn(grid) * amp)).reshape(-1)


def condition_number(op: Operator, dt: float) -> float:
    """2-norm condition number of A: A is normal (circulant), so it is max|mu| / min|mu|
    over its eigenvalues mu = 1 - dt lambda."""
    mu = np.abs(1.0 - dt * op.symbol())
    return float(mu.max() / mu.min())
