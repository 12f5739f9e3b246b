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
