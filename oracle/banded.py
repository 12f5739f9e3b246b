"""The banded preconditioner solve N^{-1} v used by Algorithm 1 before every matvec and in
the final update X = X_0 + N^{-1} Z.

The paper notes that for d = 1 (tridiagonal N) the solve is the O(n) Thomas algorithm;
wider bands are a banded LU.  Band storage throughout: band[i, p] = N(i, i + p - d)
for p = 0..2d (entries whose column falls outside [0, n) are ignored).

Cyclic band (``cyclic=True``, not in the paper): the same storage read with the column
index taken modulo n, band[i, p] = N(i, (i + p - d) mod n) -- the structure of a periodic
1D stencil, whose first and last d rows couple to the other end of the grid.  Its solve is
the plain definition: a sparse LU of the assembled matrix.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg


def _check_cyclic(n: int, d: int):
    if n < 2 * d + 1:
        raise ValueError("a cyclic band needs n >= 2d + 1 (distinct columns per row)")


def band_to_dense(band: np.ndarray, d: int, cyclic: bool = False) -> np.ndarray:
    n = band.shape[0]
    if cyclic:
        _check_cyclic(n, d)
    A = np.zeros((n, n))
    for i in range(n):
        for p in range(2 * d + 1):
            j = i + p - d
            if cyclic:
                A[i, j % n] = band[i, p]
            elif 0 <= j < n:
                A[i, j] = band[i, p]
    return A


def dense_to_band(A: np.ndarray, d: int, cyclic: bool = False) -> np.ndarray:
    n = A.shape[0]
    if cyclic:
        _check_cyclic(n, d)
    band = np.zeros((n, 2 * d + 1))
    for i in range(n):
        for p in range(2 * d + 1):
            j = i + p - d
            if cyclic:
                band[i, p] = A[i, j % n]
            elif 0 <= j < n:
                band[i, p] = A[i, j]
    return band


def transpose_band(band: np.ndarray, d: int, cyclic: bool = False) -> np.ndarray:
    """Band storage of N^T: N^T(i, i + p - d) = N(i + p - d, i) (row index modulo n for a
    cyclic band)."""
    n = band.shape[0]
    out = np.zeros_like(band)
    for i in range(n):
        for p in range(2 * d + 1):
            j = i + p - d
            if cyclic:
                out[i, p] = band[j % n, 2 * d - p]
            elif 0 <= j < n:
                out[i, p] = band[j, 2 * d - p]
    return out


def _cyclic_sparse(band: np.ndarray, d: int):
    n = band.shape[0]
    _check_cyclic(n, d)
    rows = np.repeat(np.arange(n), 2 * d + 1)
    cols = (rows + np.tile(np.arange(2 * d + 1) - d, n)) % n
    return scipy.sparse.csc_matrix((band.reshape(-1), (rows, cols)), shape=(n, n))


def solve(band: np.ndarray, d: int, v: np.ndarray, transpose: bool = False, cyclic: bool = False) -> np.ndarray:
    """N^{-1} v (or N^{-T} v): LAPACK banded LU with partial pivoting; for a cyclic band a
    sparse LU (SuperLU) of the assembled matrix."""
    if cyclic:
        S = _cyclic_sparse(np.asarray(band, dtype=np.float64), d)
        if transpose:
            S = S.T.tocsc()
        return scipy.sparse.linalg.splu(S).solve(np.asarray(v, dtype=np.float64))
    if transpose:
        band = transpose_band(band, d)
    n = band.shape[0]
    ab = np.zeros((2 * d + 1, n))
    for p in range(2 * d + 1):
        off = p - d                       # column j = i + off
        # ab[d + i - j, j] = N(i, j)  ->  ab[d - off, i + off] = band[i, p]
        lo, hi = max(0, -off), min(n, n - off)
        ab[d - off, lo + off:hi + off] = band[lo:hi, p]
    return scipy.linalg.solve_banded((d, d), ab, np.asarray(v, dtype=np.float64))


def thomas(band: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Thomas algorithm for a tridiagonal N (d = 1): forward sweep, back substitution."""
    n = band.shape[0]
    a = band[:, 0]   # N(i, i-1)
    b = band[:, 1]   # N(i, i)
    c = band[:, 2]   # N(i, i+1)
    cp = np.zeros(n)
    dp = np.zeros(n)
    cp[0] = c[0] / b[0]
    dp[0] = v[0] / b[0]
    for i in range(1, n):
        den = b[i] - a[i] * cp[i - 1]
        cp[i] = c[i] / den if i < n - 1 else 0.0
        dp[i] = (v[i] - a[i] * dp[i - 1]) / den
    x = np.zeros(n)
    x[n - 1] = dp[n - 1]
    for i in range(n - 2, -1, -1):
        x[i] = dp[i] - cp[i] * x[i + 1]
    return x
