"""Algorithm 2: MREP, the multi-regressor estimator of the banded preconditioner N.

Given the matvec history P_x, P_y (n x m: column c is one pair (x, A x)), every row of N
is a least-squares fit of P_y(i, :) on rows of P_x:

* the first d and the last d rows: a simple linear fit (beta_0, beta_1) of P_y(i, :) on
  P_x(i, :); N(i, i) = beta_1 and the intercept beta_0 is discarded;
* interior rows: the design matrix P_x* stacks a row of ones over P_x(i-d .. i+d, :)
  ((2d+2) x m: for d = 1 three regressor rows plus the intercept, four unknowns), and
  N* = (P_x* P_x*^T)^{-1} P_x* P_y(i, :)^T by the normal equations.  N*(1) is the
  intercept; N*(j) for j >= 2 multiplies P_x(i - d + j - 2, :) and goes to
  N(i, i - d + j - 2).

Readings:

* The printed scatter index N(i, i - j - d + 1) leaves the band (d = 1, j = 4 gives
  column i - 4); it is read as N(i, i - d + j - 2), the column of the regressor that
  N*(j) multiplies.
* ``intercept=False`` drops the row of ones (and the boundary intercept): a (2d+1)^2
  Gram of lagged products of P_x alone.  The paper's form is ``intercept=True``.
* ``cyclic=True`` (not in the paper): every row, the first and last d included, regresses
  on the rows i-d .. i+d taken modulo n, and the band is read cyclically
  (band[i, p] = N(i, (i + p - d) mod n)).  For a periodic 1D grid that is the structure
  of A itself, so a history that spans it recovers A exactly.
* Singular rows.  The normal equations are factored by Cholesky; a row whose relative
  pivot L_jj^2 / G_jj (the share of regressor j not explained by the ones before it)
  is <= 1e-12, or that fails to factor, is degenerate and gets the identity row
  N(i, i) = 1 with a singular flag.  The paper has no rule for this case.
"""
from __future__ import annotations

from typing import Tuple

import numpy as np
from numpy.lib.stride_tricks import sliding_window_view

REL_PIVOT = 1e-12
CHUNK = 16384


def _cholesky_solve(G: np.ndarray, rhs: np.ndarray) -> Tuple[np.ndarray, bool]:
    """Solve G beta = rhs for one SPD system; returns (beta, singular)."""
    try:
        L = np.linalg.cholesky(G)
    except np.linalg.LinAlgError:
        return np.zeros(G.shape[0]), True
    diag = np.diag(G)
    if np.any(diag <= 0.0) or np.any(np.diag(L) ** 2 <= REL_PIVOT * diag):
        return np.zeros(G.shape[0]), True
    z = np.linalg.solve(L, rhs)
    return np.linalg.solve(L.T, z), False


def _cholesky_solve_many(G: np.ndarray, rhs: np.ndarray):
    """Row-independent Cholesky solves of a stack of SPD systems (rows, q, q).

    The stack is factored at once; if any system fails to factor, each one is redone by
    itself.  Returns (solutions (rows, q), singular flags (rows,))."""
    rows, q, _ = G.shape
    try:
        L = np.linalg.cholesky(G)
    except np.linalg.LinAlgError:
        sol = np.zeros((rows, q))
        sing = np.zeros(rows, dtype=bool)
        for t in range(rows):
            sol[t], sing[t] = _cholesky_solve(G[t], rhs[t])
        return sol, sing
    diag = np.diagonal(G, axis1=1, axis2=2)
    piv = np.diagonal(L, axis1=1, axis2=2) ** 2
    sing = np.any(diag <= 0.0, axis=1) | np.any(piv <= REL_PIVOT * diag, axis=1)
    z = np.linalg.solve(L, rhs[:, :, None])
    sol = np.linalg.solve(np.transpose(L, (0, 2, 1)), z)[:, :, 0]
    sol[sing] = 0.0
    return sol, sing


def linear_fit(x: np.ndarray, y: np.ndarray, intercept: bool = True) -> Tuple[float, float, bool]:
    """Simple least-squares line y ~ beta_0 + beta_1 x; returns (beta_0, beta_1, singular)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if intercept:
        P = np.vstack([np.ones_like(x), x])
        beta, sing = _cholesky_solve(P @ P.T, P @ y)
        return float(beta[0]), float(beta[1]), sing
    P = x[None, :]
    beta, sing = _cholesky_solve(P @ P.T, P @ y)
    return 0.0, float(beta[0]), sing


def mrep(Px: np.ndarray, Py: np.ndarray, d: int, intercept: bool = True, cyclic: bool = False):
    """N in band storage band[i, p] = N(i, i + p - d) (modulo n when cyclic), and the per-row
    singular flags."""
    Px = np.asarray(Px, dtype=np.float64)
    Py = np.asarray(Py, dtype=np.float64)
    n, m = Px.shape
    if Py.shape != (n, m):
        raise ValueError("P_x and P_y must have the same shape")
    if n < 2 * d + 1:
        raise ValueError("need n >= 2d + 1 rows")
    band = np.zeros((n, 2 * d + 1))
    singular = np.zeros(n, dtype=bool)
    if cyclic:
        # every row is an interior row of the periodic grid: pad P_x with d wrapped rows on
        # each side and fit all n rows as the interior rows of the padded history
        Pad = np.concatenate([Px[n - d:], Px, Px[:d]], axis=0)
        Ypad = np.concatenate([Py[n - d:], Py, Py[:d]], axis=0)
        bp, sp = _interior(Pad, Ypad, d, intercept, band=np.zeros((n + 2 * d, 2 * d + 1)),
                           singular=np.zeros(n + 2 * d, dtype=bool))
        return bp[d:d + n], sp[d:d + n]

    # first d and last d rows: simple linear fit, N(i, i) = beta_1
    for i in list(range(d)) + list(range(n - d, n)):
        _, b1, sing = linear_fit(Px[i], Py[i], intercept)
        if sing:
            band[i, d] = 1.0
            singular[i] = True
        else:
            band[i, d] = b1

    return _interior(Px, Py, d, intercept, band, singular)


def _interior(Px, Py, d, intercept, band, singular):
    """Rows i = d .. n-d-1: regress P_y(i, :) on [1; P_x(i-d .. i+d, :)]."""
    n, m = Px.shape
    win = sliding_window_view(Px, 2 * d + 1, axis=0)      # win[r, c, j] = Px[r + j, c]
    off = 1 if intercept else 0
    q = 2 * d + 1 + off
    for r0 in range(0, n - 2 * d, CHUNK):
        r1 = min(n - 2 * d, r0 + CHUNK)
        Xs = np.transpose(win[r0:r1], (0, 2, 1))          # (rows, 2d+1, m)
        if intercept:
            Pstar = np.concatenate([np.ones((r1 - r0, 1, m)), Xs], axis=1)
        else:
            Pstar = np.ascontiguousarray(Xs)
        G = Pstar @ np.transpose(Pstar, (0, 2, 1))        # (rows, q, q)
        rhs = Pstar @ Py[d + r0:d + r1, :, None]           # (rows, q, 1)
        sol, sing = _cholesky_solve_many(G, rhs[:, :, 0])
        rows = np.arange(d + r0, d + r1)
        band[rows, :] = sol[:, off:off + 2 * d + 1]
        band[rows[sing], :] = 0.0
        band[rows[sing], d] = 1.0
        singular[rows] = sing
    return band, singular
