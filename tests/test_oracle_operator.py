"""Pins for oracle.operator and oracle.exact (Eqs. 1-4).

* The matrix-free product (periodic shifts) equals the entry-by-entry dense assembly.
* Fourier modes are eigenvectors of L with the closed-form symbols of the 2nd-order
  stencils: -4 sin^2(theta/2) / h^2 for d^2/dx^2 and i sin(theta) / h for d/dx.
* The dense LU solve of A u = u^n and the Fourier-symbol solve agree, and a single
  Fourier mode is amplified by exactly 1 / (1 - dt lambda) (implicit Euler, Eq. 3).
"""
import math

import numpy as np
import pytest

from oracle import exact
from oracle.operator import Operator


def _rand(n, seed):
    return np.random.default_rng(seed).standard_normal(n)


CASES = [
    ((12,), 4, [(1, 0, 1.0), (2, 0, 0.3)]),
    ((9, 8), 6, [(1, 0, 0.7), (1, 1, -1.3), (2, 0, 0.2), (2, 1, 0.05)]),
    ((11, 12, 13), 8, [(2, 0, 1.0), (2, 1, 0.5), (2, 2, 2.0), (4, 0, -0.01), (4, 1, -0.02), (4, 2, -0.03)]),
    ((16, 12), 2, [(3, 0, 0.4), (4, 1, -0.1)]),
]


@pytest.mark.parametrize("shape,order,terms", CASES)
def test_matrix_free_equals_dense(shape, order, terms):
    op = Operator(shape, order, terms)
    x = _rand(op.n, 1)
    L = op.dense_L()
    np.testing.assert_allclose(op.apply_L(x), L @ x, rtol=0, atol=1e-12 * np.abs(L).max() * np.abs(x).max())
    dt = 0.37
    np.testing.assert_allclose(op.apply_A(x, dt), op.dense_A(dt) @ x, rtol=0,
                               atol=1e-12 * dt * np.abs(L).max() * np.abs(x).max())


def test_direction_layout_x_fastest():
    """d/dx acts along the contiguous index; d/dy along stride nx."""
    nx, ny = 8, 6
    op = Operator((nx, ny), 2, [(1, 0, 1.0)])
    g = np.zeros((ny, nx))
    g[2, 3] = 1.0
    Lu = op.apply_L(g.reshape(-1)).reshape(ny, nx)
    h = 2 * math.pi / nx
    # (u(x+h) - u(x-h)) / 2h: the point 3 appears at x=2 with +1/2h and at x=4 with -1/2h
    assert Lu[2, 2] == pytest.approx(0.5 / h)
    assert Lu[2, 4] == pytest.approx(-0.5 / h)
    assert np.count_nonzero(Lu) == 2


@pytest.mark.parametrize("n", [8, 17, 32])
def test_symbol_closed_form_second_order(n):
    h = 2 * math.pi / n
    th = 2 * math.pi * np.arange(n) / n
    d2 = Operator((n,), 2, [(2, 0, 1.0)]).symbol_1d(0)
    np.testing.assert_allclose(d2, -4 * np.sin(th / 2) ** 2 / h ** 2, atol=1e-9)
    d1 = Operator((n,), 2, [(1, 0, 1.0)]).symbol_1d(0)
    np.testing.assert_allclose(d1, 1j * np.sin(th) / h, atol=1e-9)


@pytest.mark.parametrize("shape,order,terms", CASES)
def test_fourier_mode_is_eigenvector(shape, order, terms):
    op = Operator(shape, order, terms)
    lam = op.symbol()
    rng = np.random.default_rng(3)
    idx = tuple(int(rng.integers(0, s)) for s in reversed(shape))
    coords = np.meshgrid(*[np.arange(s) for s in reversed(shape)], indexing="ij")
    phase = sum(2 * math.pi * idx[a] * coords[a] / list(reversed(shape))[a] for a in range(len(shape)))
    mode = np.exp(1j * phase).reshape(-1)
    Lmode = op.apply_L(mode.real) + 1j * op.apply_L(mode.imag)
    np.testing.assert_allclose(Lmode, lam[idx] * mode, atol=1e-9 * (1 + abs(lam[idx])))


@pytest.mark.parametrize("shape,order,terms", CASES)
def test_dense_and_fourier_solves_agree(shape, order, terms):
    op = Operator(shape, order, terms)
    u = _rand(op.n, 5)
    dt = 0.05
    x1 = exact.solve_dense(op, u, dt)
    x2 = exact.solve_fourier(op, u, dt)
    np.testing.assert_allclose(x1, x2, rtol=0, atol=1e-11 * np.abs(x1).max())
    # and they solve A x = u
    np.testing.assert_allclose(op.apply_A(x1, dt), u, atol=1e-10 * np.abs(u).max())


def test_single_mode_amplification_closed_form():
    """u_t = nu u_xx, 2nd order: a sine mode decays by 1 / (1 + dt nu 4 sin^2(theta/2)/h^2)."""
    n, nu, dt, m = 64, 0.3, 0.2, 5
    h = 2 * math.pi / n
    x = np.arange(n) * h
    op = Operator((n,), 2, [(2, 0, nu)])
    u = np.sin(m * x)
    g = 1.0 / (1.0 + dt * nu * 4 * math.sin(m * h / 2) ** 2 / h ** 2)
    np.testing.assert_allclose(exact.solve_fourier(op, u, dt), g * u, atol=1e-13)


def test_condition_number_matches_dense():
    op = Operator((10, 6), 4, [(1, 0, 1.0), (2, 1, 0.1)])
    dt = 0.3
    s = np.linalg.svd(op.dense_A(dt), compute_uv=False)
    assert exact.condition_number(op, dt) == pytest.approx(s[0] / s[-1], rel=1e-10)
