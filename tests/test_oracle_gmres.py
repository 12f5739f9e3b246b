"""Pins for oracle.gmres (Algorithm 1) and oracle.step.

Invariants and special cases fixed by the mathematics:
* R(k) never increases within a cycle (GMRES minimises the residual over a growing space);
* V has orthonormal columns and A N^{-1} V_k = V_{k+1} H_bar_k (Arnoldi relation, right
  preconditioning);
* every stored pair satisfies P_y(:, i) = A P_x(:, i);
* the converged X equals the exact solve within the bound cond(A) * (2 tol);
* with N = I and no restart GMRES terminates in at most n iterations;
* if A - N has rank r, A N^{-1} = I + rank r and GMRES terminates in <= r + 1 iterations.
"""
import numpy as np
import pytest

from oracle import banded, exact, gmres, mrep
from oracle.operator import Operator
from oracle.step import Stepper
from paper_1308_5626_gb300 import inputs


def _problem(shape=(24,), order=4, terms=((1, 0, 1.0), (2, 0, 0.05)), dt=0.4):
    op = Operator(shape, order, terms)
    u = np.random.default_rng(11).standard_normal(op.n)
    return op, u, dt


@pytest.mark.parametrize("gs", ["mgs", "cgs2"])
@pytest.mark.parametrize("precond", [False, True])
def test_invariants(gs, precond):
    op, u, dt = _problem()
    A = op.dense_A(dt)
    band = banded.dense_to_band(A, 1) if precond else None
    Nsol = (lambda v: banded.solve(band, 1, v)) if precond else None
    res = gmres.pspgmres(lambda x: op.apply_A(x, dt), u, Nsol, 1e-13 * np.linalg.norm(u), 8, u * 0.5,
                         50, gs=gs, keep_basis=True)
    assert res.converged
    for cR in res.cycle_R:
        assert all(cR[i + 1] <= cR[i] * (1 + 1e-12) for i in range(len(cR) - 1))
    Ninv = (lambda v: banded.solve(band, 1, v)) if precond else (lambda v: v)
    for Hraw, V in zip(res.raw_H, res.V):
        k = Hraw.shape[1]
        if k == 0 or len(V) < k + 1:
            continue
        Vm = np.stack(V[:k + 1], axis=1)
        # CGS2 keeps orthogonality at rounding level; MGS loses it like eps * cond(K_k)
        assert np.abs(Vm.T @ Vm - np.eye(k + 1)).max() < (1e-12 if gs == "cgs2" else 1e-8)
        AV = np.stack([op.apply_A(Ninv(V[j]), dt) for j in range(k)], axis=1)
        assert np.abs(AV - Vm @ Hraw).max() < 1e-12 * np.abs(A).sum(axis=1).max()
    for x, y in zip(res.Px, res.Py):
        np.testing.assert_allclose(y, op.apply_A(x, dt), rtol=0, atol=1e-14)
    assert len(res.Px) == res.iterations + res.cycles
    assert res.R[-1] <= 1e-13 * np.linalg.norm(u)


def test_history_has_x0_of_every_restart():
    op, u, dt = _problem()
    x0 = u * 0.3
    res = gmres.pspgmres(lambda x: op.apply_A(x, dt), u, None, 1e-12 * np.linalg.norm(u), 4, x0, 30)
    np.testing.assert_array_equal(res.Px[0], x0)
    # the column after each cycle's m preconditioned vectors is the restart's X_0
    assert res.cycles > 1
    np.testing.assert_allclose(res.Py[5], op.apply_A(res.Px[5], dt))
    # zero initial guess: no column for the first restart
    res0 = gmres.pspgmres(lambda x: op.apply_A(x, dt), u, None, 1e-12, 4, np.zeros_like(u), 1)
    assert len(res0.Px) == res0.iterations


@pytest.mark.parametrize("shape,order,terms,dt", [
    ((64,), 4, ((1, 0, 1.0), (2, 0, 0.01)), 10 * 2 * np.pi / 64),
    ((12, 10), 6, ((1, 0, 0.8), (1, 1, 1.7), (2, 0, 0.002), (2, 1, 0.001)), 0.3),
    ((12, 12, 12), 8, ((2, 0, 1.0), (2, 1, 0.7), (2, 2, 1.5), (4, 0, -0.01), (4, 1, -0.01), (4, 2, -0.01)), 0.05),
])
def test_converges_to_exact(shape, order, terms, dt):
    op = Operator(shape, order, terms)
    u = np.random.default_rng(2).standard_normal(op.n)
    tol = 1e-10
    st = Stepper(op, b=2, m=20)
    x, info = st.step(u, dt, tol)
    assert info.converged
    ref = exact.solve_fourier(op, u, dt)
    kappa = exact.condition_number(op, dt)
    assert np.linalg.norm(x - ref) <= kappa * 2 * tol * np.linalg.norm(ref)
    # the true residual meets the tolerance up to the rounding of the update
    assert np.linalg.norm(u - op.apply_A(x, dt)) <= 2 * tol * np.linalg.norm(u)


@pytest.mark.parametrize("n", [5, 10, 16])
def test_finite_termination(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + n * np.eye(n)
    b = rng.standard_normal(n)
    res = gmres.pspgmres(lambda x: A @ x, b, None, 1e-10 * np.linalg.norm(b), n, np.zeros(n), 1)
    assert res.converged and res.iterations <= n
    np.testing.assert_allclose(res.X, np.linalg.solve(A, b), rtol=1e-8)


@pytest.mark.parametrize("r", [0, 1, 2, 3])
def test_low_rank_preconditioned_termination(r):
    n, d = 40, 2
    band = inputs.random_band(n, d, seed=r + 7)
    Nd = banded.band_to_dense(band, d)
    rng = np.random.default_rng(r)
    A = Nd + rng.standard_normal((n, r)) @ rng.standard_normal((r, n)) * 0.3
    b = rng.standard_normal(n)
    res = gmres.pspgmres(lambda x: A @ x, b, lambda v: banded.solve(band, d, v),
                         1e-9 * np.linalg.norm(b), 30, np.zeros(n), 1)
    assert res.converged and res.iterations <= r + 1


def test_mgs_and_cgs2_agree():
    op, u, dt = _problem(shape=(40,))
    outs = []
    for gs in ("mgs", "cgs2"):
        res = gmres.pspgmres(lambda x: op.apply_A(x, dt), u, None, 1e-12 * np.linalg.norm(u), 10, u, 40, gs=gs)
        outs.append(res)
    np.testing.assert_allclose(outs[0].X, outs[1].X, rtol=1e-9)
    assert abs(outs[0].iterations - outs[1].iterations) <= 1
    np.testing.assert_allclose(outs[0].R[:5], outs[1].R[:5], rtol=1e-9)


def test_progressive_preconditioner_helps_1d():
    """The paper's claim: the fitted N cuts the iteration count of the next step."""
    w = inputs.c1(256)
    op = Operator(w.shape, w.order, w.terms)
    dt = w.dt
    st = Stepper(op, b=w.b, m=w.m)
    u = w.u0
    iters = []
    for _ in range(3):
        u, info = st.step(u, dt, 1e-10)
        assert info.converged
        iters.append(info.iterations)
    assert iters[1] < iters[0] and iters[2] < iters[0], iters
