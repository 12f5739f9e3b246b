"""GPU parity of the cyclic band (psp_opts.cyclic = 1), through the C ABI.

* solve: N^{-1} v and N^{-T} v of a cyclic band (wrapped corner entries) against the
  oracle's sparse LU of the assembled matrix, FP64 1e-11 and FP32 2e-5 relative, on sizes
  from one partition level to several (ragged tails included);
* fit: every row, the wrapped first and last b included, against the oracle's cyclic MREP
  (FP64 1e-10; FP32 history against the oracle on the same rounded values);
* steps: on the 1D workload the fitted N equals A, so after the first step every FP64 step
  takes one iteration (the paper's boundary rows need up to 2b+1) and the iterates match
  the exact Fourier solve; the mixed form needs one iteration per FP32 cycle;
* a cyclic handle on a 2D grid is refused.
"""
import numpy as np
import pytest

from gpu_common import rel, t32, t64, torch_dev
from oracle import banded, exact, mrep
from oracle.operator import Operator
from paper_1308_5626_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return torch_dev()


@pytest.mark.parametrize("n,b", [(64, 1), (301, 2), (5000, 3), (70001, 4), (262144, 2)])
def test_cyclic_solve(dev, n, b):
    import torch
    from paper_1308_5626_gb300 import psp
    band = inputs.random_cyclic_band(n, b, seed=n + 11)
    v = np.random.default_rng(n).standard_normal(n)
    ref = banded.solve(band, b, v, cyclic=True)
    refT = banded.solve(band, b, v, transpose=True, cyclic=True)
    assert rel(banded.solve(band, b, v), ref) > 1e-8     # the corners matter
    s = psp.Solver((n,), 2, [(2, 0, 1.0)], b, 8, cyclic=1)
    psp.psp_set_band(s.handle, t64(band, dev))
    y = torch.empty(n, dtype=torch.float64, device=dev)
    psp.psp_apply_precond(s.handle, t64(v, dev), y)
    assert rel(y.cpu().numpy(), ref) <= 1e-11
    psp.psp_apply_precond(s.handle, t64(v, dev), y, transpose=1)
    assert rel(y.cpu().numpy(), refT) <= 1e-11
    y32 = torch.empty(n, dtype=torch.float32, device=dev)
    psp.psp_apply_precond(s.handle, t32(v, dev), y32)
    assert rel(y32.cpu().numpy(), ref) <= 2e-5
    back = torch.empty((n, 2 * b + 1), dtype=torch.float64, device=dev)
    psp.psp_get_band(s.handle, back)
    np.testing.assert_array_equal(back.cpu().numpy(), band)
    s.close()


@pytest.mark.parametrize("n,b,M,intercept", [(50, 1, 9, 1), (1000, 2, 13, 1), (4097, 4, 20, 0), (70001, 3, 16, 1)])
def test_cyclic_fit(dev, n, b, M, intercept):
    import torch
    from paper_1308_5626_gb300 import psp
    rng = np.random.default_rng(n + M)
    Px = rng.standard_normal((n, M))
    Py = rng.standard_normal((n, M))
    ref, sing = mrep.mrep(Px, Py, b, bool(intercept), cyclic=True)
    s = psp.Solver((n,), 2, [(2, 0, 1.0)], b, 8, intercept=intercept, cyclic=1)
    out = torch.empty((n, 2 * b + 1), dtype=torch.float64, device=dev)
    ns = psp.psp_fit_band(s.handle, t64(Px.T, dev), t64(Py.T, dev), out)
    assert ns == int(sing.sum()) == 0
    got = out.cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12)
    plain, _ = mrep.mrep(Px, Py, b, bool(intercept))
    assert np.abs(got[:b] - plain[:b]).max() > 1e-3     # the wrapped rows are fitted
    Px32, Py32 = Px.astype(np.float32), Py.astype(np.float32)
    ref32, _ = mrep.mrep(Px32.astype(np.float64), Py32.astype(np.float64), b, bool(intercept), cyclic=True)
    psp.psp_fit_band(s.handle, t32(Px32.T, dev), t32(Py32.T, dev), out)
    np.testing.assert_allclose(out.cpu().numpy(), ref32, rtol=1e-9, atol=1e-11)
    s.close()


@pytest.mark.parametrize("onchip", [0, 1], ids=["graphs", "onchip"])
@pytest.mark.parametrize("precision", [0, 1])
def test_cyclic_steps_one_iteration(dev, precision, onchip):
    import torch
    from paper_1308_5626_gb300 import psp
    w = inputs.c1(1024)
    op = Operator(w.shape, w.order, w.terms)
    tol = 1e-10
    its = {}
    for cyc in (0, 1):
        s = psp.Solver(w.shape, w.order, w.terms, w.b, w.m, precision=precision, cyclic=cyc, onchip=onchip)
        u = torch.tensor(w.u0, dtype=torch.float64, device=dev)
        out = torch.empty_like(u)
        seq = []
        for _ in range(5):
            ref = exact.solve_fourier(op, u.cpu().numpy(), w.dt)
            _, info = s.step(u, w.dt, tol, out=out)
            assert rel(out.cpu().numpy(), ref) <= 1e-8
            seq.append((info.iters, info.cycles))
            u, out = out, u
        its[cyc] = seq
        s.close()
    plain, cyc = its[0], its[1]
    assert plain[0][0] > 5 and cyc[0][0] == plain[0][0]        # step 1 runs with N = I
    if precision == 0:
        assert all(k == 1 for k, _ in cyc[2:]), cyc            # N = A: one iteration
    else:
        assert all(k <= c for k, c in cyc[2:]), cyc            # one iteration per FP32 cycle
    assert sum(k for k, _ in cyc[2:]) < sum(k for k, _ in plain[2:])


def test_cyclic_needs_1d(dev):
    from paper_1308_5626_gb300 import psp
    with pytest.raises(RuntimeError):
        psp.Solver((64, 64), 2, [(2, 0, 1.0)], 2, 8, cyclic=1)
    with pytest.raises(RuntimeError):
        psp.Solver((9,), 2, [(2, 0, 1.0)], 2, 8, cyclic=1)   # n < 4b + 2
