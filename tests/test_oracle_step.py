"""Pins for oracle.step: the implicit-Euler step with the progressive preconditioner.

* Every step converges to the exact Fourier solve within cond(A) * 2 tol.
* 1D (A banded within d up to the periodic corners): the fitted N is accepted and
  A N^{-1} = I + rank(2d), so every later step needs at most 2d + 1 iterations.
* Multi-dimensional grids: candidates that would slow convergence are rejected and the
  wait doubles; history is cleared when dt changes.
"""
import numpy as np
import pytest

from oracle import exact
from oracle.operator import Operator
from oracle.step import Stepper
from paper_1308_5626_gb300 import inputs


def test_1d_progressive_preconditioning_finite_termination():
    w = inputs.c1(512)
    op = Operator(w.shape, w.order, w.terms)
    st = Stepper(op, b=w.b, m=w.m)
    u = w.u0
    kappa = exact.condition_number(op, w.dt)
    for s in range(5):
        ref = exact.solve_fourier(op, u, w.dt)
        u, info = st.step(u, w.dt, w.tol)
        assert info.converged
        assert np.linalg.norm(u - ref) <= kappa * 2 * w.tol * np.linalg.norm(ref)
        if s >= 1:
            assert info.accepted and info.iterations <= 2 * w.b + 1


def test_3d_rejects_harmful_candidates_and_backs_off():
    w = inputs.c3(12, kmax=3)
    op = Operator(w.shape, w.order, w.terms)
    dt = w.with_dt(op.spectral_radius())
    st = Stepper(op, b=w.b, m=w.m)
    u = w.u0
    tried = []
    for s in range(8):
        ref = exact.solve_fourier(op, u, dt)
        u, info = st.step(u, dt, w.tol)
        assert info.converged
        assert np.linalg.norm(u - ref) <= exact.condition_number(op, dt) * 2 * w.tol * np.linalg.norm(ref)
        tried.append((info.tried_candidate, info.accepted))
    rejected = [s for s, (t, a) in enumerate(tried) if t and not a]
    assert rejected[:3] == [1, 3, 6]     # waits of 1 then 2 steps between trials


def test_history_cleared_when_dt_changes():
    w = inputs.c1(128)
    op = Operator(w.shape, w.order, w.terms)
    st = Stepper(op, b=w.b, m=w.m)
    u, info = st.step(w.u0, w.dt, w.tol)
    cols = info.hist_cols
    u, info = st.step(u, w.dt * 0.5, w.tol)
    assert not info.tried_candidate
    assert info.hist_cols <= info.iterations + info.cycles < cols + info.iterations + info.cycles


def _dense_A_band(op, dt, d, cyclic):
    """A = I - dt L of a 1D workload in band storage of half-width d (its stencil radius is
    <= d, so the cyclic band holds A exactly; the non-cyclic band drops the corner entries)."""
    from oracle import banded
    return banded.dense_to_band(op.dense_A(dt), d, cyclic=cyclic)


@pytest.mark.parametrize("cyclic", [True, False])
def test_acceptance_rule_adopts_the_operator_itself(cyclic):
    """A candidate equal to A (cyclic band: all of A; otherwise A without its periodic
    corners) is adopted by the rule: its trial cycle converges within the cycle (one
    iteration for N = A exactly; at most 2d+1 for A N^{-1} = I + rank 2d), whatever the
    reference rate of the preconditioner in use."""
    w = inputs.c1(256)
    op = Operator(w.shape, w.order, w.terms)
    st = Stepper(op, b=w.b, m=w.m, cyclic=cyclic)
    u, _ = st.step(w.u0, w.dt, w.tol)           # step 1: N = I, sets the reference rate
    st.candidate = _dense_A_band(op, w.dt, w.b, cyclic)
    st.wait = 0
    u, info = st.step(u, w.dt, w.tol)
    assert info.tried_candidate and info.accepted
    assert info.iterations <= (1 if cyclic else 2 * w.b + 1)


def test_acceptance_rule_rejects_identity_over_the_operator():
    """With N = A adopted (cyclic band, one-iteration cycles), a candidate equal to I is
    never adopted: its trial cycle reduces the residual per iteration far more slowly than
    the reference rate of N = A, and it does not converge within its cycle (the workload
    needs over 100 unpreconditioned iterations)."""
    from oracle import banded
    w = inputs.c1(256)
    op = Operator(w.shape, w.order, w.terms)
    st = Stepper(op, b=w.b, m=w.m, cyclic=True)
    u, _ = st.step(w.u0, w.dt, w.tol)
    st.candidate = _dense_A_band(op, w.dt, w.b, True)
    st.wait = 0
    u, info = st.step(u, w.dt, w.tol)
    assert info.accepted
    ident = np.zeros((w.n, 2 * w.b + 1))
    ident[:, w.b] = 1.0
    for _ in range(3):
        st.candidate = ident.copy()
        st.wait = 0
        u, info = st.step(u, w.dt, w.tol)
        assert info.tried_candidate and not info.accepted
        np.testing.assert_array_equal(st.N, _dense_A_band(op, w.dt, w.b, True))
    assert np.allclose(banded.band_to_dense(st.N, w.b, cyclic=True), op.dense_A(w.dt))


def test_without_the_rule_every_candidate_is_adopted_and_the_mock_test_stalls():
    """accept_rule=False is the paper's unconditional hand-over of N (Algorithm 1
    discussion): every fitted candidate is adopted.  On the mock test (Results section,
    restart 10, relative tolerance 1e-10) the tridiagonal fit of a seven-diagonal A then
    stalls GMRES from n = 150 (200 restarts reached), while the rule keeps every step
    converging."""
    from oracle.explicit import MatrixOperator
    for n, stalls in ((20, False), (150, True)):
        A = inputs.mock_seven_diagonal(n, seed=n)
        u = np.arange(1, n + 1, dtype=float)
        plain = Stepper(MatrixOperator(A), b=1, m=10, accept_rule=False)
        ruled = Stepper(MatrixOperator(A), b=1, m=10, accept_rule=True)
        conv_plain, conv_ruled = [], []
        for s in range(3):
            _, i1 = plain.step(u, 1.0, 1e-10)
            _, i2 = ruled.step(u, 1.0, 1e-10)
            if s >= 1:
                assert i1.tried_candidate and i1.accepted
            conv_plain.append(i1.converged)
            conv_ruled.append(i2.converged)
        assert all(conv_ruled)
        assert (not all(conv_plain)) == stalls
