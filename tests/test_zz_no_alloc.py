"""The allocation-free band fit, psp_fit_band_static, against the handle-based psp_fit_band.

psp_fit_band_static exists for callers that cannot allocate device memory (and therefore
cannot create a handle): its scratch is a static device array.  This file is collected
last so that a run stopping at its first failure has already run every other test; it
passes both alone in a fresh process and after the other tests.  Two calls in a row check
that the shared scratch left by the first call does not leak into the second.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_static_fit_matches_handle_fit_twice():
    import torch
    from gpu_common import torch_dev
    from paper_1308_5626_gb300 import psp
    dev = torch_dev()
    n, b, M = 5003, 3, 17
    s = psp.Solver((n,), 2, [(2, 0, 1.0)], b, 8)
    rng = np.random.default_rng(42)
    for call in range(2):
        Px = rng.standard_normal((M, n))
        Py = rng.standard_normal((M, n)) * (call + 1)
        if call == 1:
            Px[:, 100] = Px[:, 101]   # rows 100 and 101 identical: degenerate interior rows
        tx = torch.tensor(Px, dtype=torch.float64, device=dev)
        ty = torch.tensor(Py, dtype=torch.float64, device=dev)
        ref = torch.empty((n, 2 * b + 1), dtype=torch.float64, device=dev)
        got = torch.full((n, 2 * b + 1), float("nan"), dtype=torch.float64, device=dev)
        ns_ref = psp.psp_fit_band(s.handle, tx, ty, ref)
        ns = psp.psp_fit_band_static(tx, ty, got, b, intercept=1, stream=int(torch.cuda.current_stream().cuda_stream))
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
