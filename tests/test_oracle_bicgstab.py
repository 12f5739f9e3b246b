"""Pins of the oracle's restarted BiCGSTAB (oracle/bicgstab.py), CPU only.

* With the exact preconditioner (N = A) one iteration solves the system (p^ = A^{-1} r,
  v = r, alpha = 1, s = 0, omega = 0).
* The converged X agrees with a dense solve (and with scipy's bicgstab, an independent
  implementation) within the tolerance times the condition number; the recursive residual
  of the last iteration equals the true residual B - A X to rounding.
* Every stored pair is an exact matvec pair (P_y = A P_x), two per iteration plus the
  restart pair.
* The step driver with solver="bicgstab" reaches the exact (Fourier) solution every step,
  and on the 1D workload the adopted fitted N (A N^{-1} = I + rank 2b) cuts the iterations.
"""
import numpy as np
import pytest
import scipy.sparse.linalg

from oracle import banded, bicgstab, exact
from oracle.operator import Operator
from oracle.step import Stepper
from paper_1308_5626_gb300 import inputs


def _problem(n=96):
    op = Operator((n,), 4, [(1, 0, 1.0), (2, 0, 0.02)])
    dt = 2.0 * op.h[0]
    A = op.dense_A(dt)
    B = np.random.default_rng(5).standard_normal(n)
    return op, dt, A, B


def test_exact_preconditioner_one_iteration():
    op, dt, A, B = _problem()
    res = bicgstab.psp_bicgstab(lambda x: A @ x, B, lambda v: np.linalg.solve(A, v), 1e-12 * np.linalg.norm(B),
                                20, np.zeros_like(B), 3)
    assert res.converged and res.iterations == 1
    np.testing.assert_allclose(res.X, np.linalg.solve(A, B), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("precond", [False, True])
def test_solution_residual_and_pairs(precond):
    op, dt, A, B = _problem()
    tol = 1e-11
    eps = tol * np.linalg.norm(B)
    N = None
    if precond:
        band = banded.dense_to_band(A, 2) * (1.0 + 0.05 * np.random.default_rng(2).standard_normal((A.shape[0], 5)))
        N = lambda v: banded.solve(band, 2, v)
    res = bicgstab.psp_bicgstab(lambda x: A @ x, B, N, eps, 25, np.zeros_like(B), 50)
    assert res.converged
    ref = np.linalg.solve(A, B)
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(res.X - ref) <= 2 * kappa * tol * np.linalg.norm(ref)
    true_r = np.linalg.norm(B - A @ res.X)
    assert abs(true_r - res.R[-1]) <= 1e-9 * np.linalg.norm(B)
    for x, y in zip(res.Px, res.Py):
        np.testing.assert_allclose(y, A @ x, rtol=0, atol=1e-12 * max(1.0, np.abs(y).max()))
    assert len(res.Px) == 2 * res.iterations + (res.cycles - 1)   # restart pairs after the first
    sp, info = scipy.sparse.linalg.bicgstab(A, B, rtol=1e-13, atol=0.0, maxiter=1000)
    assert info == 0
    assert np.linalg.norm(res.X - sp) <= 4 * kappa * tol * np.linalg.norm(ref)


def test_stepper_bicgstab_steps():
    w = inputs.c1(128)
    op = Operator(w.shape, w.order, w.terms)
    st = Stepper(op, w.b, w.m, solver="bicgstab")
    u = w.u0
    its = []
    for _ in range(5):
        ref = exact.solve_fourier(op, u, w.dt)
        u_next, info = st.step(u, w.dt, 1e-10)
        assert info.converged
        assert np.linalg.norm(u_next - ref) <= 1e-8 * np.linalg.norm(ref)
        its.append(info.iterations)
        u = u_next
    assert max(its[2:]) < its[0], its
