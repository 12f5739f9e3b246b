"""One implicit-Euler step (Eq. 4) solved by Algorithm 1, with the progressive preconditioner.

The step solves A u^{n+1} = u^n with A = I - dt L.  Readings of what the paper leaves
open:

* X_0 = u^n and B = u^n; the first step runs with N = I (no fitted N exists yet).
* tol is relative: eps = tol * ||u^n|| is handed to Algorithm 1 as its absolute bound.
* The dataset grows progressively: every matvec pair of every restart is appended to
  one history that persists from step to step while dt (hence A) is unchanged, and is
  cleared when dt changes.  After each step Algorithm 2 fits a candidate N from the
  last ``max_hist`` pairs (with fewer pairs than unknowns of the fit, 2d+2 or 2d+1
  without intercept, no candidate is made).  A step that converges in a handful of
  iterations adds only a handful of pairs; a per-step history would fit N to almost
  no data.
* Acceptance of a candidate (the paper has no rule; on multi-dimensional grids the band
  fit of Krylov data can be a harmful preconditioner): the candidate preconditions the
  first restart cycle of the next step.  It is adopted if that cycle converges, or if
  its mean per-iteration residual reduction (R_end / beta)^(1/k) is no weaker than the
  reference rate of the preconditioner in use; otherwise the step continues with the
  preconditioner in use and the candidate is dropped.  After a rejection the next
  candidate waits w steps (w = 1, 2, 4, ... doubling with consecutive rejections).  The
  reference rate is that of the cycles of the last step run with the adopted
  preconditioner.
* ``cyclic=True`` (not in the paper): the fit and the solve use the cyclic band (every
  row regresses on its wrapped neighbours; see mrep and banded), the structure of A on a
  periodic 1D grid.
* ``solver="bicgstab"`` (not in the paper): the cycles are restarted BiCGSTAB
  (oracle/bicgstab.py) instead of Algorithm 1's GMRES; history, fit and acceptance are
  the same.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

from . import banded, bicgstab, gmres, mrep
from .operator import Operator


@dataclasses.dataclass
class StepInfo:
    iterations: int
    cycles: int
    converged: bool
    rel_res_est: float
    hist_cols: int
    singular_rows: int
    refit: bool
    tried_candidate: bool
    accepted: bool


def _rate(R_end: float, beta: float, k: int) -> float:
    if k <= 0 or beta <= 0.0:
        return 1.0
    return (max(R_end, 1e-300) / beta) ** (1.0 / k)


class Stepper:
    def __init__(self, op: Operator, b: int, m: int, intercept: bool = True,
                 max_restarts: int = 200, max_hist: Optional[int] = None, gs: str = "mgs",
                 accept_rule: bool = True, cyclic: bool = False, solver: str = "gmres"):
        self.op = op
        self.b = int(b)
        self.m = int(m)
        self.intercept = bool(intercept)
        self.max_restarts = int(max_restarts)
        self.max_hist = int(max_hist) if max_hist else 2 * (self.m + 1)
        self.gs = gs
        self.accept_rule = bool(accept_rule)
        self.cyclic = bool(cyclic)
        if solver not in ("gmres", "bicgstab"):
            raise ValueError("solver must be 'gmres' or 'bicgstab'")
        self.solver = solver
        self.N: Optional[np.ndarray] = None          # adopted preconditioner (None = I)
        self.candidate: Optional[np.ndarray] = None  # freshly fitted, not yet tried
        self.rate_ref: Optional[float] = None
        self.wait = 0
        self.wait_len = 1
        self.hist_x: List[np.ndarray] = []
        self.hist_y: List[np.ndarray] = []
        self.hist_dt: Optional[float] = None
        self.last: List[gmres.GmresResult] = []

    def _solver(self, band):
        if band is None:
            return None
        d = self.b
        return lambda v: banded.solve(band, d, v, cyclic=self.cyclic)

    def _cycles(self, A, B, N_solve, eps, X0, n_r):
        if self.solver == "bicgstab":
            return bicgstab.psp_bicgstab(A, B, N_solve, eps, self.m, X0, n_r)
        return gmres.pspgmres(A, B, N_solve, eps, self.m, X0, n_r, self.gs)

    def step(self, u_n: np.ndarray, dt: float, tol: float):
        u_n = np.asarray(u_n, dtype=np.float64)
        nrm = float(np.linalg.norm(u_n))
        eps = tol * nrm
        A = lambda x: self.op.apply_A(x, dt)
        if self.hist_dt != dt:
            self.hist_x, self.hist_y, self.hist_dt = [], [], dt
            self.candidate, self.rate_ref = None, None

        runs: List[gmres.GmresResult] = []
        tried = accepted = False
        X0 = u_n
        restarts_left = self.max_restarts
        if self.candidate is not None and self.wait == 0:
            tried = True
            r1 = self._cycles(A, u_n, self._solver(self.candidate), eps, X0, 1)
            runs.append(r1)
            restarts_left -= 1
            k1 = len(r1.cycle_R[0])
            rate1 = _rate(r1.cycle_R[0][-1] if k1 else r1.cycle_beta[0], r1.cycle_beta[0], k1)
            if (not self.accept_rule) or r1.converged or self.rate_ref is None or rate1 <= self.rate_ref:
                accepted = True
                self.N = self.candidate
                self.wait_len = 1
            else:
                self.wait = self.wait_len
                self.wait_len *= 2
            self.candidate = None
            X0 = r1.X
        elif self.wait > 0:
            self.wait -= 1

        main = None
        if not (runs and runs[0].converged):
            main = self._cycles(A, u_n, self._solver(self.N), eps, X0, max(restarts_left, 1))
            runs.append(main)
        self.last = runs
        X = runs[-1].X
        converged = runs[-1].converged

        # reference rate: the cycles run with the adopted preconditioner
        ref_run = main if main is not None else runs[0]
        k_tot = ref_run.iterations
        if k_tot > 0:
            R_end = ref_run.R[-1]
            self.rate_ref = _rate(R_end, ref_run.cycle_beta[0], k_tot)

        for r in runs:
            self.hist_x = (self.hist_x + r.Px)[-self.max_hist:]
            self.hist_y = (self.hist_y + r.Py)[-self.max_hist:]
        cols = len(self.hist_x)
        need = 2 * self.b + (2 if self.intercept else 1)
        sing = 0
        refit = False
        if cols >= need:
            Px = np.stack(self.hist_x, axis=1)
            Py = np.stack(self.hist_y, axis=1)
            band, flags = mrep.mrep(Px, Py, self.b, self.intercept, cyclic=self.cyclic)
            self.candidate = band
            sing = int(flags.sum())
            refit = True
        R_last = runs[-1].R[-1] if runs[-1].R else runs[-1].cycle_beta[-1]
        info = StepInfo(iterations=sum(r.iterations for r in runs),
                        cycles=sum(r.cycles for r in runs), converged=converged,
                        rel_res_est=(R_last / nrm if nrm > 0 else 0.0), hist_cols=cols,
                        singular_rows=sing, refit=refit, tried_candidate=tried,
                        accepted=accepted)
        return X, info
