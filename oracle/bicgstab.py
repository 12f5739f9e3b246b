"""Restarted right-preconditioned BiCGSTAB with the progressive history of Algorithm 1.

Test infrastructure: only the tests and the bench's CPU legs use this module.

The paper names GMRES; its preconditioner only needs matvec pairs (x, A x), which any
Krylov method produces.  This is BiCGSTAB (van der Vorst, "Bi-CGSTAB: a fast and smoothly
converging variant of Bi-CG for the solution of nonsymmetric linear systems", SIAM J. Sci.
Stat. Comput. 1992) with right preconditioning, restarted from the true residual every
n_it iterations like Algorithm 1's cycles, recording the same history:

* restart: store (X_0, A X_0), r = B - A X_0, beta = ||r||, shadow residual rh = r,
  rho = rh . r;
* iteration k: p = r (k = 0) or p = r + (rho / rho_prev)(alpha / omega)(p - omega v);
  p^ = N^{-1} p, v = A p^ (stored pair); alpha = rho / (rh . v); s = r - alpha v;
  s^ = N^{-1} s, t = A s^ (stored pair); omega = (t . s) / (t . t) (0 when t = 0);
  X += alpha p^ + omega s^; r = s - omega t; R(k) = ||r||; rho_prev = rho, rho = rh . r;
  the cycle ends when R(k) <= eps (finish), or on a breakdown (rh . v = 0, rho = 0 or
  omega = 0; the next restart takes a fresh shadow residual).

Readings: the method's stopping test uses the recursive residual r (as GMRES uses R(k));
a restart recomputes the true residual.  No early exit on ||s||: the second pair of the
iteration is always formed (with s = 0 it is (0, 0) and omega = 0).  Both pairs of
iteration k are stored scaled by sigma = 1 / ||r|| (r at the start of the iteration): a
multiple of a matvec pair is a matvec pair, and BiCGSTAB's directions shrink with the
residual (to 1e-11 in a converged cycle), which left unscaled makes the per-row designs of
Algorithm 2 ill-conditioned (condition 4e9 on the 1D workload); GMRES's pairs are
normalised by construction.
"""
from __future__ import annotations

from typing import Callable, List, Optional

import numpy as np

from .gmres import GmresResult


def psp_bicgstab(apply_A: Callable[[np.ndarray], np.ndarray], B: np.ndarray,
                 N_solve: Optional[Callable[[np.ndarray], np.ndarray]], eps: float,
                 n_it: int, X0: np.ndarray, n_r: int) -> GmresResult:
    Nsol = N_solve if N_solve is not None else (lambda v: v.copy())
    B = np.asarray(B, dtype=np.float64)
    X = np.asarray(X0, dtype=np.float64).copy()
    Px: List[np.ndarray] = []
    Py: List[np.ndarray] = []
    R_all: List[float] = []
    cycle_R: List[List[float]] = []
    cycle_beta: List[float] = []
    iterations = cycles = 0
    finish = False
    for _l in range(n_r):
        cycles += 1
        if np.any(X != 0.0):
            Px.append(X.copy())
            Py.append(apply_A(X))
            r = B - Py[-1]
        else:
            r = B.copy()
        beta = float(np.linalg.norm(r))
        cycle_beta.append(beta)
        cR: List[float] = []
        if beta <= eps:
            finish = True
            cycle_R.append(cR)
            break
        rh = r.copy()
        rho = float(rh @ r)
        p = np.zeros_like(r)
        v = np.zeros_like(r)
        alpha = omega = 1.0
        for k in range(n_it):
            if k == 0:
                p = r.copy()
            else:
                p = r + (rho / rho_prev) * (alpha / omega) * (p - omega * v)
            # the stored pairs are scaled by 1 / ||r||: the directions shrink with the
            # residual, and unscaled columns would make the fit's designs ill-conditioned
            sig = 1.0 / float(np.linalg.norm(r))
            ph = Nsol(p)
            v = apply_A(ph)
            Px.append(sig * ph)
            Py.append(sig * v)
            iterations += 1
            rv = float(rh @ v)
            alpha = rho / rv if rv != 0.0 else 0.0
            s = r - alpha * v
            sh = Nsol(s)
            t = apply_A(sh)
            Px.append(sig * sh)
            Py.append(sig * t)
            tt = float(t @ t)
            omega = float(t @ s) / tt if tt != 0.0 else 0.0
            X = X + alpha * ph + omega * sh
            r = s - omega * t
            Rk = float(np.linalg.norm(r))
            cR.append(Rk)
            R_all.append(Rk)
            rho_prev, rho = rho, float(rh @ r)
            if Rk <= eps:
                finish = True
                break
            if rv == 0.0 or omega == 0.0 or rho == 0.0:
                break
        cycle_R.append(cR)
        if finish:
            break
    return GmresResult(X=X, R=R_all, cycle_R=cycle_R, cycle_beta=cycle_beta, Px=Px, Py=Py,
                       iterations=iterations, cycles=cycles, converged=finish, raw_H=[], V=[])
