"""The paper's mock test (Results section) on the GPU: an explicit seven-diagonal A through
psp_create_banded, against the oracle's step driver on the same matrix.

* psp_matvec applies A (and A^T on an adjoint handle) to 1e-14 of the row scale.
* Three steps of u^n = (1..n) with d = 1 and restart 10 (step 1: N = I; then the fitted
  tridiagonal N is tried and kept or dropped by the acceptance rule): every step reaches
  the dense solution within kappa * 2 tol, its iteration count follows the oracle's within
  max(2, 10%) (20% on a step that tries a candidate), and the tried/accepted flags agree.
"""
import numpy as np
import pytest

from gpu_common import rel, t64, torch_dev
from oracle.explicit import MatrixOperator
from oracle.step import Stepper
from paper_1308_5626_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return torch_dev()


def test_banded_matvec_and_adjoint(dev):
    import torch
    from paper_1308_5626_gb300 import psp
    n = 333
    A = inputs.mock_seven_diagonal(n, seed=4)
    band = t64(inputs.dense_to_band(A, 3).reshape(-1), dev)
    x = np.random.default_rng(5).standard_normal(n)
    for adj, M in ((0, A), (1, A.T)):
        s = psp.Solver.banded(band, 3, 1, 10, adjoint=adj)
        y = torch.empty(n, dtype=torch.float64, device=dev)
        psp.psp_matvec(s.handle, t64(x, dev), y, 1.0)
        scale = np.abs(A).sum(axis=1).max() * np.abs(x).max()
        assert np.abs(y.cpu().numpy() - M @ x).max() <= 1e-14 * scale
        s.close()


@pytest.mark.parametrize("onchip", [0, 1], ids=["graphs", "onchip"])
@pytest.mark.parametrize("n", inputs.MOCK_SIZES)
def test_mock_steps_follow_the_oracle(dev, n, onchip):
    from paper_1308_5626_gb300 import psp
    A = inputs.mock_seven_diagonal(n, seed=n)
    u = np.arange(1.0, n + 1.0)
    ref = np.linalg.solve(A, u)
    kappa = np.linalg.cond(A)
    tol = 1e-10
    s = psp.Solver.banded(t64(inputs.dense_to_band(A, 3).reshape(-1), dev), 3, 1, 10, onchip=onchip)
    st = Stepper(MatrixOperator(A), b=1, m=10)
    for step in range(3):
        x_o, oinfo = st.step(u, 1.0, tol)
        x, info = s.step(t64(u, dev), 1.0, tol)
        assert info.status == 0
        assert rel(x.cpu().numpy(), ref) <= kappa * 2 * tol, (step, rel(x.cpu().numpy(), ref))
        slack = oinfo.iterations // 5 if oinfo.tried_candidate else oinfo.iterations // 10
        assert abs(info.iters - oinfo.iterations) <= max(2, slack), (step, info.iters, oinfo.iterations)
        assert bool(info.flags & psp.PSP_FLAG_CANDIDATE_TRIED) == oinfo.tried_candidate, step
        assert bool(info.flags & psp.PSP_FLAG_CANDIDATE_ACCEPTED) == oinfo.accepted, step
    s.close()
