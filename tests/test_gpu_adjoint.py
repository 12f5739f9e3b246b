"""GPU parity of the adjoint path (the differentiable step), through the C ABI.

* The adjoint handle's operator is A^T: its matvec equals the assembled A^T x (a
  non-symmetric operator, so A^T != A), FP64 1e-13 of the rounding scale.
* psp_apply_L gives L x and every term's unit-alpha derivative D_t x (oracle stencils).
* psp_apply_precond(transpose=1) solves N^T y = v (LAPACK banded solve of N^T).
* Gradients of ||u^T - target||^2 through T steps w.r.t. u^0, dt and the term coefficients
  match the oracle's dense adjoint chain on a 32 x 32 copy of the 2D diffusion workload
  within 1e-6 relative, in the FP64 and the mixed form.
* On the full 512 x 512 workload (10 steps), the FP64 gradients w.r.t. the two
  coefficients and dt match central finite differences of the GPU forward (h = 1e-6
  relative) within 1e-6 relative, and a checkpointed rollout gives the same gradients.
"""
import numpy as np
import pytest

from gpu_common import rel, t64, torch_dev
from oracle import adjoint, banded
from oracle.operator import Operator
from paper_1308_5626_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return torch_dev()


def _scale(op, dt, x):
    return (1 + dt * sum(abs(a) * op.h[d] ** -k * sum(abs(w) for w in op.weights[(k, op.order)])
                         for k, d, a in op.terms)) * np.abs(x).max()


@pytest.mark.parametrize("shape,order,terms", [
    ((200,), 4, [(1, 0, 1.0), (2, 0, 0.01)]),
    ((40, 36), 6, [(1, 0, 0.8), (1, 1, -1.3), (2, 0, 1e-3), (2, 1, 2e-3)]),
])
def test_adjoint_handle_applies_transpose(dev, shape, order, terms):
    import torch
    from paper_1308_5626_gb300 import psp
    op = Operator(shape, order, terms)
    dt = 0.37 * min(op.h)
    x = np.random.default_rng(2).standard_normal(op.n)
    ref = op.dense_A(dt).T @ x
    s = psp.Solver(shape, order, terms, 2, 8, adjoint=1)
    y = torch.empty(op.n, dtype=torch.float64, device=dev)
    psp.psp_matvec(s.handle, t64(x, dev), y, dt)
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-13 * _scale(op, dt, x)
    assert np.abs(op.dense_A(dt) @ x - ref).max() > 1e-3 * np.abs(ref).max()
    s.close()


def test_apply_L_and_terms(dev):
    import torch
    from paper_1308_5626_gb300 import psp
    shape, order = (48, 40), 6
    terms = [(1, 0, 0.8), (2, 1, 2e-3), (2, 0, 1e-3)]
    op = Operator(shape, order, terms)
    x = np.random.default_rng(3).standard_normal(op.n)
    s = psp.Solver(shape, order, terms, 2, 8)
    y = torch.empty(op.n, dtype=torch.float64, device=dev)
    psp.psp_apply_L(s.handle, -1, t64(x, dev), y)
    ref = op.apply_L(x)
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    for t in range(len(terms)):
        psp.psp_apply_L(s.handle, t, t64(x, dev), y)
        ref = adjoint.apply_term(op, t, x)
        assert np.abs(y.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max(), t
    # the matvec still uses A after psp_apply_L changed the shared coefficient block
    psp.psp_matvec(s.handle, t64(x, dev), y, 0.01)
    assert np.abs(y.cpu().numpy() - op.apply_A(x, 0.01)).max() <= 1e-12 * _scale(op, 0.01, x)
    s.close()


@pytest.mark.parametrize("n,b", [(300, 2), (5000, 3), (70001, 4)])
def test_transposed_preconditioner_solve(dev, n, b):
    import torch
    from paper_1308_5626_gb300 import psp
    band = inputs.random_band(n, b, seed=n + 7)
    v = np.random.default_rng(n).standard_normal(n)
    ref = banded.solve(band, b, v, transpose=True)
    s = psp.Solver((n,), 2, [(2, 0, 1.0)], b, 8)
    psp.psp_set_band(s.handle, t64(band, dev))
    y = torch.empty(n, dtype=torch.float64, device=dev)
    psp.psp_apply_precond(s.handle, t64(v, dev), y, transpose=1)
    assert rel(y.cpu().numpy(), ref) <= 1e-11
    psp.psp_apply_precond(s.handle, t64(v, dev), y, transpose=0)
    assert rel(y.cpu().numpy(), banded.solve(band, b, v)) <= 1e-11
    s.close()


def _c5_problem(n, precision, tol):
    from paper_1308_5626_gb300 import autograd
    w, factors = inputs.c5(n)
    op_true = Operator(w.shape, w.order, w.terms)
    dt = w.with_dt(op_true.spectral_radius())
    alphas = np.array([t.alpha for t in w.terms]) * factors
    prob = autograd.Problem(w.shape, w.order, [(t.k, t.dir) for t in w.terms], w.b, w.m,
                            precision=precision, tol=tol)
    return w, op_true, dt, alphas, prob


@pytest.mark.parametrize("precision", [0, 1])
def test_gradients_match_dense_adjoint(dev, precision):
    import torch
    from paper_1308_5626_gb300 import autograd
    steps = 4
    tol = 1e-13 if precision == 0 else 1e-10
    w, op_true, dt, alphas, prob = _c5_problem(32, precision, tol)
    target = adjoint.rollout(op_true, w.u0, dt, steps)[-1]
    op = adjoint.with_alphas(op_true, alphas)
    ref = adjoint.rollout_gradients(op, w.u0, dt, steps, target)
    u0 = torch.tensor(w.u0, dtype=torch.float64, device=dev, requires_grad=True)
    dtt = torch.tensor(dt, dtype=torch.float64, device=dev, requires_grad=True)
    al = torch.tensor(alphas, dtype=torch.float64, device=dev, requires_grad=True)
    uT = autograd.rollout(u0, dtt, al, prob, steps)
    loss = ((uT - torch.tensor(target, device=dev)) ** 2).sum()
    loss.backward()
    assert abs(loss.item() - ref.loss) <= 1e-8 * ref.loss
    assert rel(u0.grad.cpu().numpy(), ref.du0) <= 1e-6
    assert abs(dtt.grad.item() - ref.ddt) <= 1e-6 * abs(ref.ddt)
    np.testing.assert_allclose(al.grad.cpu().numpy(), ref.dalpha, rtol=1e-6)
    prob.close()


def test_full_size_gradients_match_finite_differences(dev):
    """512 x 512, 10 steps, FP64: dLoss/dalpha (2) and dLoss/d dt against central
    differences of the GPU forward; a checkpointed rollout reproduces the gradients."""
    import torch
    from paper_1308_5626_gb300 import autograd
    steps = 10
    w, op_true, dt, alphas, prob = _c5_problem(512, 0, 1e-13)
    target = torch.tensor(adjoint_target(op_true, w.u0, dt, steps), device=dev)

    def loss_of(al_np, dt_v):
        with torch.no_grad():
            u = autograd.rollout(torch.tensor(w.u0, dtype=torch.float64, device=dev),
                                 torch.tensor(dt_v, dtype=torch.float64, device=dev),
                                 torch.tensor(al_np, dtype=torch.float64, device=dev), prob, steps)
            return float(((u - target) ** 2).sum())

    grads = []
    for ck in (False, True):
        u0 = torch.tensor(w.u0, dtype=torch.float64, device=dev, requires_grad=True)
        dtt = torch.tensor(dt, dtype=torch.float64, device=dev, requires_grad=True)
        al = torch.tensor(alphas, dtype=torch.float64, device=dev, requires_grad=True)
        uT = autograd.rollout(u0, dtt, al, prob, steps, checkpoint=ck)
        ((uT - target) ** 2).sum().backward()
        grads.append((al.grad.cpu().numpy().copy(), dtt.grad.item()))
    np.testing.assert_allclose(grads[1][0], grads[0][0], rtol=1e-8)
    assert abs(grads[1][1] - grads[0][1]) <= 1e-8 * abs(grads[0][1])
    dal, ddt = grads[0]
    for t in range(2):
        h = 1e-6 * alphas[t]
        ap, am = alphas.copy(), alphas.copy()
        ap[t] += h
        am[t] -= h
        fd = (loss_of(ap, dt) - loss_of(am, dt)) / (2 * h)
        assert abs(fd - dal[t]) <= 1e-6 * abs(fd), (t, fd, dal[t])
    h = 1e-6 * dt
    fd = (loss_of(alphas, dt + h) - loss_of(alphas, dt - h)) / (2 * h)
    assert abs(fd - ddt) <= 1e-6 * abs(fd), (fd, ddt)
    prob.close()


def adjoint_target(op, u0, dt, steps):
    """u^steps with the true coefficients, by the oracle's exact (Fourier) steps."""
    from oracle import exact
    u = u0
    for _ in range(steps):
        u = exact.solve_fourier(op, u, dt)
    return u


@pytest.mark.parametrize("shape,order,terms", [
    ((300,), 4, [(1, 0, 1.0), (2, 0, 0.01)]),
    ((40, 36), 6, [(1, 0, 0.8), (1, 1, -1.3), (2, 0, 1e-3), (2, 1, 2e-3)]),
    ((16, 12, 20), 8, [(2, 0, 0.7), (2, 1, 1.1), (2, 2, 1.9), (4, 0, -1e-3), (4, 1, -1e-3), (4, 2, -2e-3)]),
])
def test_adjoint_grads_match_the_oracle_terms(dev, shape, order, terms):
    """psp_adjoint_grads: dLoss/d dt = lambda . L u and dLoss/d alpha_t = dt lambda . D_t u,
    against the oracle's stencils (each term applied alone with unit alpha), 1e-12 of the
    products' rounding scale sum|lambda| |D_t| |u|."""
    from paper_1308_5626_gb300 import psp
    op = Operator(shape, order, terms)
    rng = np.random.default_rng(11)
    lam, u = rng.standard_normal(op.n), rng.standard_normal(op.n)
    dt = 0.3 * min(op.h)
    s = psp.Solver(shape, order, terms, 2, 8)
    g = psp.psp_adjoint_grads(s.handle, t64(lam, dev), t64(u, dev), dt, len(terms))
    s.close()
    d = []
    for (k, dd, a) in terms:
        d.append(float(lam @ Operator(shape, order, [(k, dd, 1.0)]).apply_L(u)))
    scale = [float(np.abs(lam) @ np.abs(Operator(shape, order, [(k, dd, 1.0)]).apply_L(u))) + 1.0
             for (k, dd, a) in terms]
    for t, (k, dd, a) in enumerate(terms):
        assert abs(g[1 + t] - dt * d[t]) <= 1e-12 * dt * scale[t] * 100
    ref0 = sum(a * dv for (k, dd, a), dv in zip(terms, d))
    assert abs(g[0] - ref0) <= 1e-12 * sum(abs(a) * sc for (k, dd, a), sc in zip(terms, scale)) * 100


def test_adjoint_grads_refuse_adjoint_and_banded_handles(dev):
    import torch
    from paper_1308_5626_gb300 import psp
    x = torch.zeros(64, dtype=torch.float64, device=dev)
    Ab = t64(inputs.dense_to_band(np.eye(64) * 2.0, 1), dev).reshape(-1)
    for s in (psp.Solver((64,), 2, [(2, 0, 1.0)], 2, 8, adjoint=1), psp.Solver.banded(Ab, 1, 1, 8)):
        with pytest.raises(psp.PspError) as e:
            psp.psp_adjoint_grads(s.handle, x, x, 0.1, 1)
        assert e.value.status == psp.PSP_ERR_ARG
        s.close()


@pytest.mark.parametrize("cyclic", [0, 1])
def test_set_band_from_hands_over_the_transpose(dev, cyclic):
    """psp_set_band_from(dst, src, 1): dst adopts N^T of src's adopted N (the oracle's
    transpose_band of the same band, cyclic too); with transpose = 0, N itself; from a handle
    with no adopted N, the identity."""
    import torch
    from paper_1308_5626_gb300 import psp
    n, b = 257, 3
    band = inputs.random_cyclic_band(n, b, seed=5) if cyclic else inputs.random_band(n, b, seed=5)
    src = psp.Solver((n,), 4, [(2, 0, 1.0)], b, 8, cyclic=cyclic)
    dst = psp.Solver((n,), 4, [(2, 0, 1.0)], b, 8, cyclic=cyclic, adjoint=1)
    out = torch.empty((n, 2 * b + 1), dtype=torch.float64, device=dev)
    psp.psp_set_band_from(dst.handle, src.handle, 1)
    psp.psp_get_band(dst.handle, out)
    ident = np.zeros((n, 2 * b + 1))
    ident[:, b] = 1.0
    np.testing.assert_array_equal(out.cpu().numpy(), ident)
    psp.psp_set_band(src.handle, t64(band, dev))
    psp.psp_set_band_from(dst.handle, src.handle, 1)
    psp.psp_get_band(dst.handle, out)
    np.testing.assert_array_equal(out.cpu().numpy(), banded.transpose_band(band, b, cyclic=bool(cyclic)))
    psp.psp_set_band_from(dst.handle, src.handle, 0)
    psp.psp_get_band(dst.handle, out)
    np.testing.assert_array_equal(out.cpu().numpy(), band)
    src.close()
    dst.close()
