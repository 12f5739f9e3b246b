"""Higher-order implicit integrators built from the implicit step (Eq. 4).

Test infrastructure: only the tests and the bench's CPU legs use this module.

The paper advances with implicit Euler, whose building block is one solve of
(I - dt L) x = rhs.  Two classical second-order integrators reuse exactly that solve, with
another right-hand side and a scaled time step (not in the paper):

* BDF2 (two-step backward differentiation):
      (I - 2/3 dt L) u^{n+1} = (4 u^n - u^{n-1}) / 3,
  started from u^0 and u^1 (one implicit-Euler step gives u^1).
* SDIRK2 (Alexander's two-stage, stiffly accurate, L-stable singly diagonally implicit
  Runge-Kutta method, gamma = 1 - 1/sqrt(2)):
      (I - gamma dt L) U1 = u^n
      (I - gamma dt L) U2 = u^n + (1 - gamma) dt L U1
      u^{n+1} = U2.
  Both stages solve with the same matrix, so one preconditioner serves both.

The solves are the plain definition of the step (exact.solve_fourier for periodic
constant-coefficient grids, or a dense solve).
"""
from __future__ import annotations

import math
from typing import Callable, List

import numpy as np

from . import exact
from .operator import Operator

GAMMA = 1.0 - 1.0 / math.sqrt(2.0)

Solve = Callable[[Operator, np.ndarray, float], np.ndarray]


def _arr(x) -> np.ndarray:
    """float64 array (complex input kept complex, for single Fourier modes)."""
    a = np.asarray(x)
    return a if np.iscomplexobj(a) else a.astype(np.float64, copy=False)


def bdf2_rhs(u_n: np.ndarray, u_nm1: np.ndarray) -> np.ndarray:
    return (4.0 * _arr(u_n) - _arr(u_nm1)) / 3.0


def bdf2_step(op: Operator, u_nm1: np.ndarray, u_n: np.ndarray, dt: float,
              solve: Solve = exact.solve_fourier) -> np.ndarray:
    """u^{n+1} of BDF2: the implicit step with dt' = 2 dt / 3 on (4 u^n - u^{n-1}) / 3."""
    return solve(op, bdf2_rhs(u_n, u_nm1), 2.0 * dt / 3.0)


def sdirk2_step(op: Operator, u_n: np.ndarray, dt: float, solve: Solve = exact.solve_fourier) -> np.ndarray:
    """u^{n+1} of the two-stage SDIRK method (both stages: the implicit step with gamma dt)."""
    u_n = _arr(u_n)
    U1 = solve(op, u_n, GAMMA * dt)
    rhs2 = u_n + (1.0 - GAMMA) * dt * op.apply_L(U1)
    return solve(op, rhs2, GAMMA * dt)


def rollout(op: Operator, u0: np.ndarray, dt: float, steps: int, method: str,
            solve: Solve = exact.solve_fourier) -> List[np.ndarray]:
    """u^0 .. u^steps; method 'euler', 'bdf2' (first step implicit Euler) or 'sdirk2'."""
    us = [_arr(u0)]
    for s in range(steps):
        if method == "euler" or (method == "bdf2" and s == 0):
            us.append(solve(op, us[-1], dt))
        elif method == "bdf2":
            us.append(bdf2_step(op, us[-2], us[-1], dt, solve))
        elif method == "sdirk2":
            us.append(sdirk2_step(op, us[-1], dt, solve))
        else:
            raise ValueError("unknown method " + method)
    return us
