"""Algorithm 1: the Progressive Statistical Preconditioned GMRES (PSPGMRES) with restarts.

Written in the algorithm's own order and notation:

* for each restart l = 1..n_r: store P_x(:, i) = X_0 and P_y(:, i) = A X_0; form the
  residual R_bar = B - P_y(:, i), V(:, 1) = R_bar / ||R_bar||, G(1) = ||R_bar||;
* for k = 1..n_A: G(k+1) = 0; Y_k = N^{-1} V(:, k) (right preconditioning); store
  P_x(:, i) = Y_k, P_y(:, i) = A Y_k; U_k = P_y(:, i); Gram-Schmidt against V(:, 1..k)
  filling H(1..k, k); H(k+1, k) = ||U_k||; V(:, k+1) = U_k / H(k+1, k); apply the old
  Givens rotations to column k, form the new rotation (gamma, C(k), S(k)), rotate G,
  R(k) = |G(k+1)|; stop the cycle with the finish flag when R(k) <= eps;
* Q = H^{-1} G on the completed k x k triangle, Z = sum_j Q(j) V(:, j),
  X = X_0 + N^{-1} Z, X_0 = X; leave when the finish flag is set.

Readings of passages the paper leaves open:

* Gram-Schmidt: the paper's loop is modified Gram-Schmidt (``gs="mgs"``).  ``gs="cgs2"``
  is classical Gram-Schmidt applied twice, equal in exact arithmetic.
* Z_k starts at zero; Q solves the leading k x k upper triangle of the rotated H.
* eps is an absolute bound on R(k) as printed; callers pass tol * ||B|| for a
  relative tolerance.
* Breakdown: when H(k+1, k) <= 1e-14 * ||U_k|| (U_k before orthogonalisation) the
  Krylov space is invariant; V(:, k+1) is not formed and the cycle ends after the
  Givens step (the finish flag follows R(k) <= eps as usual).
* History columns are numbered across restarts and include X_0 of every restart.  A
  restart whose X_0 is exactly zero stores no column (its matvec is skipped: A 0 = 0).
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional

import numpy as np

BREAKDOWN_REL = 1e-14


@dataclasses.dataclass
class GmresResult:
    X: np.ndarray
    R: List[float]                  # R(k) of every iteration, all cycles in order
    cycle_R: List[List[float]]      # R(k) per cycle
    cycle_beta: List[float]         # ||R_bar|| at the start of every cycle
    Px: List[np.ndarray]
    Py: List[np.ndarray]
    iterations: int                 # Arnoldi iterations (preconditioned matvecs)
    cycles: int
    converged: bool
    raw_H: List[np.ndarray]         # per cycle: H before rotations, (k+1) x k
    V: List[List[np.ndarray]]       # per cycle: the basis V(:, 1..k+1)


def pspgmres(apply_A: Callable[[np.ndarray], np.ndarray], B: np.ndarray,
             N_solve: Optional[Callable[[np.ndarray], np.ndarray]], eps: float,
             n_A: int, X0: np.ndarray, n_r: int, gs: str = "mgs",
             keep_basis: bool = False) -> GmresResult:
    if gs not in ("mgs", "cgs2"):
        raise ValueError("gs must be 'mgs' or 'cgs2'")
    Nsol = N_solve if N_solve is not None else (lambda v: v.copy())
    B = np.asarray(B, dtype=np.float64)
    X0 = np.asarray(X0, dtype=np.float64).copy()
    X = X0.copy()
    Px: List[np.ndarray] = []
    Py: List[np.ndarray] = []
    R_all: List[float] = []
    cycle_R: List[List[float]] = []
    cycle_beta: List[float] = []
    raw_H: List[np.ndarray] = []
    bases: List[List[np.ndarray]] = []
    iterations = 0
    cycles = 0
    finish = False

    for _l in range(n_r):
        cycles += 1
        if np.any(X0 != 0.0):
            Px.append(X0.copy())
            Py.append(apply_A(X0))
            Rbar = B - Py[-1]
        else:
            Rbar = B.copy()
        beta = float(np.linalg.norm(Rbar))
        cycle_beta.append(beta)
        cR: List[float] = []
        if beta == 0.0:
            finish = True
            cycle_R.append(cR)
            raw_H.append(np.zeros((1, 0)))
            bases.append([])
            break
        V = [Rbar / beta]
        G = np.zeros(n_A + 1)
        G[0] = beta
        H = np.zeros((n_A + 1, n_A))
        Hraw = np.zeros((n_A + 1, n_A))
        C = np.zeros(n_A)
        S = np.zeros(n_A)
        k_done = 0
        for k in range(n_A):                      # the paper's k = 1..n_A, 0-based here
            G[k + 1] = 0.0
            Y = Nsol(V[k])
            Px.append(Y)
            Py.append(apply_A(Y))
            U = Py[-1].copy()
            iterations += 1
            u_norm0 = float(np.linalg.norm(U))
            if gs == "mgs":
                for j in range(k + 1):
                    H[j, k] = float(np.dot(V[j], U))
                    U = U - H[j, k] * V[j]
            else:
                h1 = np.array([float(np.dot(V[j], U)) for j in range(k + 1)])
                for j in range(k + 1):
                    U = U - h1[j] * V[j]
                h2 = np.array([float(np.dot(V[j], U)) for j in range(k + 1)])
                for j in range(k + 1):
                    U = U - h2[j] * V[j]
                H[:k + 1, k] = h1 + h2
            H[k + 1, k] = float(np.linalg.norm(U))
            Hraw[:k + 2, k] = H[:k + 2, k]
            breakdown = H[k + 1, k] <= BREAKDOWN_REL * u_norm0
            if not breakdown:
                V.append(U / H[k + 1, k])
            for j in range(k):                    # old rotations j = 1..k-1
                delta = H[j, k]
                H[j, k] = delta * C[j] + S[j] * H[j + 1, k]
                H[j + 1, k] = -delta * S[j] + C[j] * H[j + 1, k]
            gamma = float(np.hypot(H[k, k], H[k + 1, k]))
            C[k] = H[k, k] / gamma
            S[k] = H[k + 1, k] / gamma
            H[k, k] = gamma
            H[k + 1, k] = 0.0
            delta = G[k]
            G[k] = C[k] * delta + S[k] * G[k + 1]
            G[k + 1] = -S[k] * delta + C[k] * G[k + 1]
            Rk = abs(G[k + 1])
            cR.append(Rk)
            R_all.append(Rk)
            k_done = k + 1
            if Rk <= eps:
                finish = True
                break
            if breakdown:
                break
        cycle_R.append(cR)
        raw_H.append(Hraw[:k_done + 1, :k_done].copy())
        bases.append(V if keep_basis else [])
        # Q = H^{-1} G on the completed triangle (back substitution)
        Q = np.zeros(k_done)
        for j in range(k_done - 1, -1, -1):
            Q[j] = (G[j] - float(np.dot(H[j, j + 1:k_done], Q[j + 1:k_done]))) / H[j, j]
        Z = np.zeros_like(B)
        for j in range(k_done):
            Z = Z + Q[j] * V[j]
        X = X0 + Nsol(Z)
        X0 = X.copy()
        if finish:
            break

    return GmresResult(X=X, R=R_all, cycle_R=cycle_R, cycle_beta=cycle_beta, Px=Px, Py=Py,
                       iterations=iterations, cycles=cycles, converged=finish,
                       raw_H=raw_H, V=bases)
