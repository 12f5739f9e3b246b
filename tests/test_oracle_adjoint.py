"""Pins of the oracle's adjoint gradients (oracle/adjoint.py), CPU only.

The gradients of ||u^T - target||^2 through T implicit-Euler steps are checked against
central finite differences of the oracle's own dense forward rollout (a different
computation: no adjoint solve, no per-term operators), for a random direction in u^0, for
dt and for every term coefficient.  A mistake in a sign, a transposition or a missing dt
factor fails one of them.
"""
import numpy as np
import pytest

from oracle import adjoint
from oracle.operator import Operator


def _case(shape, terms, order=6, steps=3, seed=0):
    op = Operator(shape, order, terms)
    rng = np.random.default_rng(seed)
    u0 = rng.standard_normal(op.n)
    target = rng.standard_normal(op.n) * 0.1
    dt = 2.0 / max(1e-12, np.abs(op.symbol()).max())
    return op, u0, target, dt, steps


CASES = [
    ((24,), 6, [(2, 0, 0.8), (1, 0, 0.3)]),
    ((12, 10), 6, [(2, 0, 1.1e-1), (2, 1, 0.7e-1)]),
    ((8, 8, 9), 4, [(2, 0, 0.5), (2, 2, 0.9), (4, 1, -1e-3)]),
]


@pytest.mark.parametrize("shape,order,terms", CASES)
def test_adjoint_matches_finite_differences(shape, order, terms):
    op, u0, target, dt, steps = _case(shape, terms, order=order)
    gr = adjoint.rollout_gradients(op, u0, dt, steps, target)
    assert abs(gr.loss - adjoint.loss(op, u0, dt, steps, target)) <= 1e-12 * gr.loss
    # u^0 along a random direction
    v = np.random.default_rng(1).standard_normal(op.n)
    h = 1e-6
    fd = (adjoint.loss(op, u0 + h * v, dt, steps, target) - adjoint.loss(op, u0 - h * v, dt, steps, target)) / (2 * h)
    assert abs(fd - gr.du0 @ v) <= 1e-6 * max(1.0, abs(fd))
    # dt
    hd = 1e-6 * dt
    fd = (adjoint.loss(op, u0, dt + hd, steps, target) - adjoint.loss(op, u0, dt - hd, steps, target)) / (2 * hd)
    assert abs(fd - gr.ddt) <= 1e-6 * max(1.0, abs(fd))
    # each term coefficient
    alphas = np.array([a for _, _, a in op.terms])
    for t in range(len(alphas)):
        ha = 1e-6 * abs(alphas[t])
        ap, am = alphas.copy(), alphas.copy()
        ap[t] += ha
        am[t] -= ha
        fd = (adjoint.loss(adjoint.with_alphas(op, ap), u0, dt, steps, target)
              - adjoint.loss(adjoint.with_alphas(op, am), u0, dt, steps, target)) / (2 * ha)
        assert abs(fd - gr.dalpha[t]) <= 1e-6 * max(1.0, abs(fd)), (t, fd, gr.dalpha[t])


def test_apply_term_sums_to_L():
    op = Operator((10, 9), 4, [(2, 0, 0.7), (1, 1, -0.4), (2, 1, 1.3)])
    u = np.random.default_rng(3).standard_normal(op.n)
    total = sum(a * adjoint.apply_term(op, t, u) for t, (_, _, a) in enumerate(op.terms))
    np.testing.assert_allclose(total, op.apply_L(u), rtol=1e-13, atol=1e-13 * np.abs(op.apply_L(u)).max())


def test_adjoint_state_is_transpose_solve():
    """For a non-symmetric operator (an advection term) A^T differs from A: the adjoint
    state must use A^T (checked against the Fourier solve with the conjugate symbol, whose
    eigenvalues are those of A^T on the periodic grid)."""
    op = Operator((16,), 4, [(1, 0, 1.0), (2, 0, 0.05)])
    dt = 0.3
    g = np.random.default_rng(4).standard_normal(op.n)
    lam = np.linalg.solve(op.dense_A(dt).T, g)
    amp = 1.0 / (1.0 - dt * np.conj(op.symbol()))
    lam_f = np.real(np.fft.ifft(np.fft.fft(g) * amp))
    np.testing.assert_allclose(lam, lam_f, rtol=1e-12, atol=1e-12)
    assert np.abs(np.linalg.solve(op.dense_A(dt), g) - lam).max() > 1e-3
