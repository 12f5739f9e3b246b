"""GPU parity of the integrators built on the step (psp_step_bdf2, psp_step_sdirk2), through
the C ABI, against the oracle's integrators with exact (Fourier) solves:

* BDF2 (started by one implicit-Euler psp_step) and the two-stage SDIRK method, 5 steps of
  the 1D workload (n = 256) and of a 48 x 40 copy of the 2D workload, FP64 (tol 1e-12:
  within 2e-9 relative of the oracle at every step) and mixed (tol 1e-10: within 1e-7);
* the SDIRK stages share the handle's history: the second stage of a step and the later
  steps run preconditioned once a candidate is adopted (1D: fewer iterations than step 1);
* an explicit banded operator handle is refused (the integrators scale L by dt).
"""
import numpy as np
import pytest

from gpu_common import rel, torch_dev
from oracle import integrators
from oracle.operator import Operator
from paper_1308_5626_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return torch_dev()


def _workloads():
    return [inputs.c1(256), inputs.c2(48, 40)]


@pytest.mark.parametrize("wi", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("method", ["bdf2", "sdirk2"])
def test_integrator_matches_oracle(dev, wi, precision, method):
    import torch
    from paper_1308_5626_gb300 import psp
    w = _workloads()[wi]
    op = Operator(w.shape, w.order, w.terms)
    tol, bound = (1e-12, 2e-9) if precision == 0 else (1e-10, 1e-7)
    ref = integrators.rollout(op, w.u0, w.dt, 5, method)
    s = psp.Solver(w.shape, w.order, w.terms, w.b, w.m, precision=precision)
    us = [torch.tensor(w.u0, dtype=torch.float64, device=dev)]
    its = []
    for k in range(5):
        out = torch.empty_like(us[-1])
        if method == "bdf2" and k == 0:
            _, info = s.step(us[-1], w.dt, tol, out=out)
        elif method == "bdf2":
            _, info = s.step_bdf2(us[-2], us[-1], w.dt, tol, out=out)
        else:
            _, info = s.step_sdirk2(us[-1], w.dt, tol, out=out)
        us.append(out)
        its.append(int(info.iters))
        assert rel(out.cpu().numpy(), ref[k + 1]) <= bound, (k, rel(out.cpu().numpy(), ref[k + 1]))
    if wi == 0 and method == "sdirk2" and precision == 0:
        assert its[-1] < its[0], its          # the stages share the progressive preconditioner
    s.close()


def test_integrators_refuse_banded_handles(dev):
    import torch
    from paper_1308_5626_gb300 import psp
    n = 50
    band = torch.tensor(inputs.dense_to_band(inputs.mock_seven_diagonal(n, seed=n), 3).reshape(-1),
                        dtype=torch.float64, device=dev)
    s = psp.Solver.banded(band, 3, 1, 10)
    u = torch.ones(n, dtype=torch.float64, device=dev)
    with pytest.raises(RuntimeError):
        s.step_sdirk2(u, 0.1, 1e-10)
    with pytest.raises(RuntimeError):
        s.step_bdf2(u, u, 0.1, 1e-10)
    s.close()
