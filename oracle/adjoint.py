"""Gradients of a loss through implicit-Euler steps (Eq. 4), by the adjoint of the step.

Test infrastructure: only the tests and the bench's CPU legs use this module.

One step solves A u^{n+1} = u^n with A = I - dt L and L = sum_t alpha_t D_t (Eqs. 1-2, D_t
the central difference of term t scaled by h^-k).  Differentiating A u^{n+1} = u^n gives
A du^{n+1} = du^n + d(dt) L u^{n+1} + dt sum_t d(alpha_t) D_t u^{n+1}, so for a loss with
g = dLoss/du^{n+1} and the adjoint state lambda = A^{-T} g:

    dLoss/du^n = lambda,  dLoss/d(dt) = lambda . L u^{n+1},  dLoss/d(alpha_t) = dt lambda . D_t u^{n+1}.

The paper has no adjoint; this is the derivative of its step, written with the assembled A
(tiny grids: the plain definition) and chained backwards over a rollout.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Sequence

import numpy as np

from .operator import Operator


def apply_term(op: Operator, t: int, u: np.ndarray) -> np.ndarray:
    """D_t u: term t of the operator with unit alpha (h_dir^-k times its central difference)."""
    k, d, _ = op.terms[t]
    one = Operator(op.shape, op.order, [(k, d, 1.0)])
    return one.apply_L(u)


def with_alphas(op: Operator, alphas: Sequence[float]) -> Operator:
    """The same operator with the term coefficients replaced."""
    return Operator(op.shape, op.order, [(k, d, float(a)) for (k, d, _), a in zip(op.terms, alphas)])


def rollout(op: Operator, u0: np.ndarray, dt: float, steps: int) -> List[np.ndarray]:
    """u^0, u^1, ..., u^steps by dense solves of A (Eq. 4)."""
    A = op.dense_A(dt)
    us = [np.asarray(u0, dtype=np.float64)]
    for _ in range(steps):
        us.append(np.linalg.solve(A, us[-1]))
    return us


def loss(op: Operator, u0: np.ndarray, dt: float, steps: int, target: np.ndarray) -> float:
    """||u^steps - target||^2."""
    u = rollout(op, u0, dt, steps)[-1]
    r = u - target
    return float(r @ r)


@dataclass
class Gradients:
    du0: np.ndarray
    ddt: float
    dalpha: np.ndarray
    loss: float


def rollout_gradients(op: Operator, u0: np.ndarray, dt: float, steps: int, target: np.ndarray) -> Gradients:
    """Gradients of ||u^steps - target||^2 w.r.t. u^0, dt and the term coefficients, by the
    adjoint chain: g_steps = 2 (u^steps - target); per step backwards lambda = A^{-T} g,
    accumulate the dt and alpha terms at u^{s+1}, and pass g_s = lambda on."""
    us = rollout(op, u0, dt, steps)
    AT = op.dense_A(dt).T
    g = 2.0 * (us[-1] - target)
    ddt = 0.0
    dalpha = np.zeros(len(op.terms))
    for s in range(steps - 1, -1, -1):
        lam = np.linalg.solve(AT, g)
        u1 = us[s + 1]
        ddt += float(lam @ op.apply_L(u1))
        for t in range(len(op.terms)):
            dalpha[t] += dt * float(lam @ apply_term(op, t, u1))
        g = lam
    r = us[-1] - target
    return Gradients(du0=g, ddt=ddt, dalpha=dalpha, loss=float(r @ r))
