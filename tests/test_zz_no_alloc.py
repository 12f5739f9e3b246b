"""The allocation-free band fit, psp_fit_band_static, against the handle-based psp_fit_band.

psp_fit_band_static exists for callers that cannot allocate device memory (and therefore
cannot create a handle): its scratch is a static device array.  This file is collected
last so that a run stopping at its first failure has already run every other test; it
passes both alone in a fresh process and after the other tests.  Two calls in a row check
that the shared scratch left by the first call does not leak into the second; the cases
cover both half-widths at the ends of the range (the per-row moment stride 4b+4 differs
from the array's fixed 4*4+4 sizing), both intercept modes, a leading dimension larger
than n, and the largest accepted n, which fills the static array.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = [
    # (n, ld, b, intercept, M)
    (5003, 5003, 3, 1, 17),
    (4099, 4099, 1, 0, 9),
    (4099, 4099, 1, 1, 9),
    (3001, 3001, 4, 0, 21),
    (3001, 3001, 4, 1, 21),
    (2500, 2560, 2, 1, 13),     # ld > n
    (65536, 65536, 4, 1, 12),   # the largest accepted n: the whole static array
]


@pytest.mark.parametrize("n,ld,b,intercept,M", CASES)
def test_static_fit_matches_handle_fit_twice(n, ld, b, intercept, M):
    import torch
    from gpu_common import torch_dev
    from paper_1308_5626_gb300 import psp
    dev = torch_dev()
    s = psp.Solver((n,), 2, [(2, 0, 1.0)], b, 8, intercept=intercept)
    rng = np.random.default_rng(42 + n + b)
    stream = int(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        Px = rng.standard_normal((M, ld))
        Py = rng.standard_normal((M, ld)) * (call + 1)
        if call == 1:
            Px[:, 100] = Px[:, 101]   # rows 100 and 101 identical: degenerate interior rows
        tx = torch.tensor(Px, dtype=torch.float64, device=dev)
        ty = torch.tensor(Py, dtype=torch.float64, device=dev)
        ref = torch.empty((n, 2 * b + 1), dtype=torch.float64, device=dev)
        got = torch.full((n, 2 * b + 1), float("nan"), dtype=torch.float64, device=dev)
        ns_ref = psp.psp_fit_band(s.handle, tx, ty, ref)
        ns = psp.psp_fit_band_static(tx, ty, got, b, intercept=intercept, n=n, stream=stream)
        torch.cuda.synchronize()
        assert ns == ns_ref
        if call == 1:
            assert ns > 0
        np.testing.assert_allclose(got.cpu().numpy(), ref.cpu().numpy(), rtol=1e-12, atol=1e-14)
    s.close()


def test_static_fit_rejects_oversized_input():
    import torch
    from gpu_common import torch_dev
    from paper_1308_5626_gb300 import psp
    dev = torch_dev()
    n = 65537
    x = torch.zeros((2, n), dtype=torch.float64, device=dev)
    out = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    with pytest.raises(psp.PspError) as e:
        psp.psp_fit_band_static(x, x, out, 1)
    assert e.value.status == psp.PSP_ERR_ARG
    assert "65536" in str(e.value)


def test_static_fit_refuses_other_dtypes_and_short_output():
    """FP32 history (which psp_fit_band would route to its FP32 entry) and an output too
    small for n (2b+1) values are refused by the binding before any pointer is passed."""
    import torch
    from gpu_common import torch_dev
    from paper_1308_5626_gb300 import psp
    dev = torch_dev()
    n, b = 1000, 2
    x32 = torch.zeros((4, n), dtype=torch.float32, device=dev)
    x64 = torch.zeros((4, n), dtype=torch.float64, device=dev)
    out = torch.zeros((n, 2 * b + 1), dtype=torch.float64, device=dev)
    for args in ((x32, x32, out), (x64, x64, out[:-1]), (x64, x64.t(), out)):
        with pytest.raises(psp.PspError) as e:
            psp.psp_fit_band_static(*args, b)
        assert e.value.status == psp.PSP_ERR_ARG
