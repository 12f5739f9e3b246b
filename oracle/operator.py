"""The semi-discrete operator L (Eqs. 1-2) and the implicit-Euler matrix A = I - dt L (Eq. 4).

Periodic grid with n_i points per direction, h_i = 2 pi / n_i, vectors flattened with
x fastest.  L u = sum over terms alpha * h_dir^-k * sum_j w_j u(x + j h e_dir) with the
central weights of ``oracle.fd``.  The matrix-free product (a residual evaluation that
stands in for A x in the paper's matrix-free GMRES) uses periodic shifts; ``dense_L``
assembles the same operator entry by entry for tiny grids.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np

from . import fd


class Operator:
    def __init__(self, shape: Sequence[int], order: int, terms: Sequence) -> None:
        self.shape = tuple(int(s) for s in shape)
        self.ndim = len(self.shape)
        self.order = int(order)
        self.h = tuple(2.0 * math.pi / s for s in self.shape)
        # terms: objects or tuples with (k, dir, alpha)
        self.terms: List[Tuple[int, int, float]] = []
        for t in terms:
            if hasattr(t, "k"):
                self.terms.append((int(t.k), int(t.dir), float(t.alpha)))
            else:
                k, d, a = t
                self.terms.append((int(k), int(d), float(a)))
        for k, d, _ in self.terms:
            if not 0 <= d < self.ndim:
                raise ValueError("term direction out of range")
            if 2 * fd.half_width(k, self.order) + 1 > self.shape[d]:
                raise ValueError("stencil wider than the grid")
        self.weights = {(k, self.order): fd.central_weights(k, self.order) for k, _, _ in self.terms}

    @property
    def n(self) -> int:
        return int(np.prod(self.shape))

    def _axis(self, d: int) -> int:
        # array viewed as (n_{ndim-1}, ..., n_1, n_0): direction d is axis ndim-1-d
        return self.ndim - 1 - d

    def apply_L(self, u: np.ndarray) -> np.ndarray:
        """L u, matrix-free, with periodic shifts."""
        grid = np.asarray(u, dtype=np.float64).reshape(tuple(reversed(self.shape)))
        out = np.zeros_like(grid)
        for k, d, alpha in self.terms:
            w = self.weights[(k, self.order)]
            r = (len(w) - 1) // 2
            scale = alpha * self.h[d] ** (-k)
            ax = self._axis(d)
            for j in range(-r, r + 1):
                if w[j + r] != 0.0:
                    # u(x + j h): element i takes the value at i + j
                    out += (scale * w[j + r]) * np.roll(grid, -j, axis=ax)
        return out.reshape(-1)

    def apply_A(self, u: np.ndarray, dt: float) -> np.ndarray:
        """A u = u - dt L u (Eq. 4)."""
        u = np.asarray(u, dtype=np.float64)
        return u - dt * self.apply_L(u)

    def dense_L(self) -> np.ndarray:
        """L assembled entry by entry (tiny grids only)."""
        n = self.n
        if n > 4096:
            raise ValueError("dense assembly is for tiny grids")
        L = np.zeros((n, n))
        strides = [1]
        for s in self.shape[:-1]:
            strides.append(strides[-1] * s)
        for idx in range(n):
            coord = [(idx // strides[d]) % self.shape[d] for d in range(self.ndim)]
            for k, d, alpha in self.terms:
                w = self.weights[(k, self.order)]
                r = (len(w) - 1) // 2
                scale = alpha * self.h[d] ** (-k)
                for j in range(-r, r + 1):
                    c = list(coord)
                    c[d] = (c[d] + j) % self.shape[d]
                    col = sum(c[q] * strides[q] for q in range(self.ndim))
                    L[idx, col] += scale * w[j + r]
        return L

    def dense_A(self, dt: float) -> np.ndarray:
        return np.eye(self.n) - dt * self.dense_L()

    def symbol_1d(self, d: int) -> np.ndarray:
        """Per-direction symbol lambda_d(theta_m), theta_m = 2 pi m / n_d, m = 0..n_d-1.

        A Fourier mode exp(i theta . x / h) is an eigenvector of L with eigenvalue
        sum_d lambda_d(theta_d).
        """
        nd = self.shape[d]
        theta = 2.0 * math.pi * np.arange(nd) / nd
        lam = np.zeros(nd, dtype=np.complex128)
        for k, dd, alpha in self.terms:
            if dd != d:
                continue
            w = self.weights[(k, self.order)]
            r = (len(w) - 1) // 2
            scale = alpha * self.h[d] ** (-k)
            for j in range(-r, r + 1):
                lam += scale * w[j + r] * np.exp(1j * j * theta)
        return lam

    def symbol(self) -> np.ndarray:
        """Eigenvalues of L on the grid's Fourier modes, array shaped (n_{ndim-1}, ..., n_0)."""
        lam = np.zeros(tuple(reversed(self.shape)), dtype=np.complex128)
        for d in range(self.ndim):
            shp = [1] * self.ndim
            shp[self._axis(d)] = self.shape[d]
            lam = lam + self.symbol_1d(d).reshape(shp)
        return lam

    def spectral_radius(self) -> float:
        """max |lambda| of L over the grid's Fourier modes."""
        return float(np.abs(self.symbol()).max())
