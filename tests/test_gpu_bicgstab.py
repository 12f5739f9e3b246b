"""GPU parity of the BiCGSTAB solver (psp_opts.solver = PSP_SOLVER_BICGSTAB), through the
C ABI, against the oracle's restarted BiCGSTAB step driver (oracle/bicgstab.py) and the
exact (Fourier) solve:

* 1D workload (n = 256), FP64, tol 1e-12, 5 steps: every step within 2e-9 relative of the
  exact solve; the same candidate decisions (tried / accepted) as the oracle's driver; the
  iterations of the steps after the first match the oracle's within one (the fitted N
  built from BiCGSTAB's scaled pairs gives A N^{-1} = I + rank 2b);
* a 48 x 40 copy of the 2D workload, FP64, 3 steps, within 2e-9 of the exact solve;
* the solver is refused in the mixed form and for m < 3.
"""
import numpy as np
import pytest

from gpu_common import rel, torch_dev
from oracle import exact
from oracle.operator import Operator
from oracle.step import Stepper
from paper_1308_5626_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return torch_dev()


def _run(dev, w, steps, tol):
    import torch
    from paper_1308_5626_gb300 import psp
    op = Operator(w.shape, w.order, w.terms)
    s = psp.Solver(w.shape, w.order, w.terms, w.b, w.m, solver=psp.PSP_SOLVER_BICGSTAB)
    u = torch.tensor(w.u0, dtype=torch.float64, device=dev)
    out = torch.empty_like(u)
    rows = []
    for _ in range(steps):
        ref = exact.solve_fourier(op, u.cpu().numpy(), w.dt)
        _, info = s.step(u, w.dt, tol, out=out)
        assert rel(out.cpu().numpy(), ref) <= 2e-9
        rows.append((int(info.iters), bool(info.flags & psp.PSP_FLAG_CANDIDATE_TRIED),
                     bool(info.flags & psp.PSP_FLAG_CANDIDATE_ACCEPTED)))
        u, out = out, u
    s.close()
    return rows


def test_bicgstab_1d_matches_oracle_driver(dev):
    w = inputs.c1(256)
    tol = 1e-12
    gpu = _run(dev, w, 5, tol)
    op = Operator(w.shape, w.order, w.terms)
    st = Stepper(op, w.b, w.m, solver="bicgstab")
    u = w.u0
    ora = []
    for _ in range(5):
        u, info = st.step(u, w.dt, tol)
        ora.append((info.iterations, info.tried_candidate, info.accepted))
    assert [g[1:] for g in gpu] == [o[1:] for o in ora], (gpu, ora)
    for g, o in zip(gpu[1:], ora[1:]):
        assert abs(g[0] - o[0]) <= 1, (gpu, ora)
    assert max(g[0] for g in gpu[2:]) <= 2 * w.b + 2


def test_bicgstab_2d(dev):
    w = inputs.c2(48, 40)
    _run(dev, w, 3, 1e-12)


def test_bicgstab_options(dev):
    from paper_1308_5626_gb300 import psp
    with pytest.raises(RuntimeError):
        psp.Solver((64,), 2, [(2, 0, 1.0)], 2, 8, precision=psp.PSP_MIXED, solver=psp.PSP_SOLVER_BICGSTAB)
    with pytest.raises(RuntimeError):
        psp.Solver((64,), 2, [(2, 0, 1.0)], 2, 2, solver=psp.PSP_SOLVER_BICGSTAB)


def test_bicgstab_with_cyclic_band(dev):
    """BiCGSTAB with the cyclic band on the 1D workload: the fitted N equals A, so after the
    step that adopts it every FP64 step takes one iteration and matches the exact solve."""
    import torch
    from paper_1308_5626_gb300 import psp
    w = inputs.c1(1024)
    op = Operator(w.shape, w.order, w.terms)
    s = psp.Solver(w.shape, w.order, w.terms, w.b, w.m, solver=psp.PSP_SOLVER_BICGSTAB, cyclic=1)
    u = torch.tensor(w.u0, dtype=torch.float64, device=dev)
    out = torch.empty_like(u)
    its = []
    for _ in range(5):
        ref = exact.solve_fourier(op, u.cpu().numpy(), w.dt)
        _, info = s.step(u, w.dt, 1e-12, out=out)
        assert rel(out.cpu().numpy(), ref) <= 2e-9
        its.append(int(info.iters))
        u, out = out, u
    s.close()
    assert its[0] > 5 and all(k == 1 for k in its[2:]), its
