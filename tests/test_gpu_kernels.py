"""GPU parity of the kernels taken one at a time, through the C ABI, against the oracle.

* matvec (stencil): FP64 within 1e-13 of the oracle's matrix-free product (relative to
  sum |coef| * max |x|, the rounding scale of the sum); FP32 within 2e-6 of that scale.
* band solve: y = N^{-1} v against LAPACK's banded LU; FP64 within 1e-12 * cond-scale,
  FP32 within 1e-5, for b = 1..4 on sizes from one group to many levels with ragged tails.
* band fit (Algorithm 2): against the oracle's MREP on well-conditioned random histories
  within 1e-10, FP32 histories within 1e-9 (the fit is FP64 either way), exact recovery
  of a banded A, and degenerate rows flagged and set to the identity row.
"""
import numpy as np
import pytest

from gpu_common import rel, t32, t64, torch_dev
from oracle import banded, mrep
from oracle.operator import Operator
from paper_1308_5626_gb300 import inputs

pytestmark = pytest.mark.gpu

STENCIL_CASES = [
    ((1000,), 4, [(1, 0, 1.0), (2, 0, 0.01)]),
    ((67, 45), 6, [(1, 0, 0.8), (1, 1, 1.3), (2, 0, 1e-3), (2, 1, 2e-3)]),
    ((24, 20, 18), 8, [(2, 0, 1.0), (2, 1, 0.6), (2, 2, 1.7), (4, 0, -1e-4), (4, 1, -2e-4), (4, 2, -3e-4)]),
    ((33, 17, 12), 2, [(3, 0, 0.3), (1, 2, -0.5), (4, 1, 0.01)]),
    ((1024, 1024), 6, [(1, 0, 0.8), (1, 1, 1.3), (2, 0, 1e-3), (2, 1, 2e-3)]),
    # 3D grids that take the z-marching tiled kernel (x a whole number of 32-vector tiles in
    # FP32 and FP64, y a multiple of 8 rows): one tile, several tiles and z chunks, and the
    # smallest z extent (2R + 1 planes)
    ((128, 16, 12), 8, [(2, 0, 1.0), (2, 1, 0.6), (2, 2, 1.7), (4, 0, -1e-4), (4, 1, -2e-4), (4, 2, -3e-4)]),
    ((256, 24, 20), 6, [(2, 0, 0.9), (1, 1, 0.4), (2, 2, 1.1), (1, 2, -0.7)]),
    ((128, 16, 11), 8, [(4, 0, -2e-4), (2, 1, 0.8), (4, 2, -1e-4)]),
]


@pytest.fixture(scope="module")
def dev():
    return torch_dev()


def _handle(shape, order, terms, b=2, m=8, precision=0):
    from paper_1308_5626_gb300 import psp
    return psp.Solver(shape, order, terms, b, m, precision=precision)


@pytest.mark.parametrize("shape,order,terms", STENCIL_CASES)
def test_matvec(dev, shape, order, terms):
    import torch
    from paper_1308_5626_gb300 import psp
    op = Operator(shape, order, terms)
    dt = 0.37 * min(op.h) ** 2
    x = np.random.default_rng(1).standard_normal(op.n)
    ref = op.apply_A(x, dt)
    s = _handle(shape, order, terms)
    y = torch.empty(op.n, dtype=torch.float64, device=dev)
    psp.psp_matvec(s.handle, t64(x, dev), y, dt)
    scale = (1 + dt * sum(abs(a) * op.h[d] ** -k * sum(abs(w) for w in op.weights[(k, order)])
                          for k, d, a in op.terms)) * np.abs(x).max()
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-13 * scale
    y32 = torch.empty(op.n, dtype=torch.float32, device=dev)
    psp.psp_matvec(s.handle, t32(x, dev), y32, dt)
    assert np.abs(y32.cpu().numpy().astype(np.float64) - ref).max() <= 2e-6 * scale
    s.close()


def test_matvec_3d_full_size(dev):
    """The 256^3 grid of the 3D workload (8th order, radius 5): the whole product against
    the oracle's matrix-free stencil, FP64 and FP32, at the same rounding-scale bounds."""
    import torch
    from paper_1308_5626_gb300 import psp
    w = inputs.c3(256, with_u0=False)
    op = Operator(w.shape, w.order, w.terms)
    dt = 1e-3
    x = np.random.default_rng(11).standard_normal(op.n)
    ref = op.apply_A(x, dt)
    s = psp.Solver(w.shape, w.order, w.terms, w.b, 2, max_hist_cols=4)
    y = torch.empty(op.n, dtype=torch.float64, device=dev)
    psp.psp_matvec(s.handle, t64(x, dev), y, dt)
    scale = (1 + dt * sum(abs(a) * op.h[d] ** -k * sum(abs(v) for v in op.weights[(k, w.order)])
                          for k, d, a in op.terms)) * np.abs(x).max()
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-13 * scale
    y32 = torch.empty(op.n, dtype=torch.float32, device=dev)
    psp.psp_matvec(s.handle, t32(x, dev), y32, dt)
    assert np.abs(y32.cpu().numpy().astype(np.float64) - ref).max() <= 2e-6 * scale
    s.close()


def test_stencil_weights_match_oracle(dev):
    from paper_1308_5626_gb300 import psp
    shape, order, terms = STENCIL_CASES[2]
    op = Operator(shape, order, terms)
    s = _handle(shape, order, terms)
    w, R = psp.psp_get_stencil(s.handle)
    for d in range(3):
        ref = np.zeros(2 * R + 1)
        for k, dd, a in op.terms:
            if dd == d:
                ww = op.weights[(k, order)]
                r = (len(ww) - 1) // 2
                ref[R - r:R + r + 1] += a * op.h[d] ** -k * np.array(ww)
        np.testing.assert_allclose(w[d], ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    s.close()


BAND_CASES = [(5, 1), (9, 2), (64, 3), (200, 4), (1000, 1), (4099, 2), (70001, 3), (70003, 4), (1 << 20, 4)]


@pytest.mark.parametrize("n,b", BAND_CASES)
@pytest.mark.parametrize("kind", ["dominant", "pd_part"])
def test_band_solve(dev, n, b, kind):
    import torch
    from paper_1308_5626_gb300 import psp
    band = inputs.random_band(n, b, seed=n + b) if kind == "dominant" else inputs.random_pd_part_band(n, b, seed=n)
    v = np.random.default_rng(n).standard_normal(n)
    ref = banded.solve(band, b, v)
    s = _handle((n,), 2, [(2, 0, 1.0)], b=b)
    psp.psp_set_band(s.handle, t64(band, dev))
    y = torch.empty(n, dtype=torch.float64, device=dev)
    psp.psp_apply_precond(s.handle, t64(v, dev), y)
    assert rel(y.cpu().numpy(), ref) <= 1e-11
    y32 = torch.empty(n, dtype=torch.float32, device=dev)
    psp.psp_apply_precond(s.handle, t32(v, dev), y32)
    assert rel(y32.cpu().numpy(), ref) <= 2e-5
    # in place, and the stored band comes back unchanged
    vv = t64(v, dev)
    psp.psp_apply_precond(s.handle, vv, vv)
    assert rel(vv.cpu().numpy(), ref) <= 1e-11
    out = torch.empty((n, 2 * b + 1), dtype=torch.float64, device=dev)
    psp.psp_get_band(s.handle, out)
    np.testing.assert_array_equal(out.cpu().numpy(), band)
    s.close()


def test_singular_band_is_rejected(dev):
    from paper_1308_5626_gb300 import psp
    n, b = 100, 2
    band = inputs.random_band(n, b, seed=3)
    band[40:60, :] = 0.0
    s = _handle((n,), 2, [(2, 0, 1.0)], b=b)
    with pytest.raises(psp.PspError) as e:
        psp.psp_set_band(s.handle, t64(band, dev))
    assert e.value.status == psp.PSP_ERR_NUMERIC
    s.close()


@pytest.mark.parametrize("n,b,M", [(40, 1, 12), (300, 2, 20), (5000, 3, 17), (70001, 4, 33)])
@pytest.mark.parametrize("intercept", [1, 0])
def test_fit_random(dev, n, b, M, intercept):
    import torch
    from paper_1308_5626_gb300 import psp
    rng = np.random.default_rng(n + M)
    Px = rng.standard_normal((n, M))
    Py = rng.standard_normal((n, M))
    ref, sing = mrep.mrep(Px, Py, b, bool(intercept))
    s = psp.Solver((n,), 2, [(2, 0, 1.0)], b, 8, intercept=intercept)
    out = torch.empty((n, 2 * b + 1), dtype=torch.float64, device=dev)
    ns = psp.psp_fit_band(s.handle, t64(Px.T, dev), t64(Py.T, dev), out)
    assert ns == int(sing.sum()) == 0
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-10, atol=1e-12)
    # FP32 history: the oracle sees the same rounded values
    Px32, Py32 = Px.astype(np.float32), Py.astype(np.float32)
    ref32, _ = mrep.mrep(Px32.astype(np.float64), Py32.astype(np.float64), b, bool(intercept))
    psp.psp_fit_band(s.handle, t32(Px32.T, dev), t32(Py32.T, dev), out)
    np.testing.assert_allclose(out.cpu().numpy(), ref32, rtol=1e-9, atol=1e-11)
    s.close()


def test_fit_fp32_history_wide_range(dev):
    """FP32 history whose rows span 1e-18 .. 1e18 (every product of two entries stays a normal
    FP32 value, as the double-float moments need; neighbouring rows 36 decades apart give Gram
    matrices far outside FP32's range, which the FP64 row solves take): against the oracle, per
    row within 1e-9 plus the row's Gram condition number times 50 M 2^-46 (the moments'
    double-float rounding)."""
    import torch
    from paper_1308_5626_gb300 import psp
    n, b, M = 3000, 3, 21
    rng = np.random.default_rng(77)
    scale = 10.0 ** rng.uniform(-18, 18, size=n)
    scale[1000:1010] = 1e-18
    scale[1010:1020] = 1e18
    Px = (rng.standard_normal((n, M)) * scale[:, None]).astype(np.float32)
    Py = (rng.standard_normal((n, M)) * scale[:, None]).astype(np.float32)
    ref, sing = mrep.mrep(Px.astype(np.float64), Py.astype(np.float64), b, True)
    s = psp.Solver((n,), 2, [(2, 0, 1.0)], b, 8)
    out = torch.empty((n, 2 * b + 1), dtype=torch.float64, device=dev)
    ns = psp.psp_fit_band(s.handle, t32(Px.T, dev), t32(Py.T, dev), out)
    assert ns == int(sing.sum())
    got = out.cpu().numpy()
    for i in range(b, n - b):
        P = np.vstack([np.ones(M), Px[i - b:i + b + 1].astype(np.float64)])
        tol = 1e-9 + 50 * M * 2.0 ** -46 * np.linalg.cond(P @ P.T)
        err = np.abs(got[i] - ref[i]).max() / max(np.abs(ref[i]).max(), 1e-300)
        assert err <= tol, (i, err, tol)
    s.close()


def test_fit_ld_and_exact_recovery(dev):
    import torch
    from paper_1308_5626_gb300 import psp
    n, b, M, ld = 3001, 3, 15, 3072
    A = banded.band_to_dense(inputs.random_band(n, b, seed=9), b) if n < 4000 else None
    Px = inputs.random_history(n, M, seed=2)
    Py = A @ Px
    pad = np.zeros((M, ld))
    pady = np.zeros((M, ld))
    pad[:, :n] = Px.T
    pady[:, :n] = Py.T
    s = psp.Solver((n,), 2, [(2, 0, 1.0)], b, 8)
    out = torch.empty((n, 2 * b + 1), dtype=torch.float64, device=dev)
    psp.psp_fit_band(s.handle, t64(pad, dev), t64(pady, dev), out, ld=ld, M=M)
    got = out.cpu().numpy()
    Ab = banded.dense_to_band(A, b)
    np.testing.assert_allclose(got[b:n - b], Ab[b:n - b], atol=1e-9 * np.abs(Ab).max())
    s.close()


def test_fit_degenerate_rows(dev):
    import torch
    from paper_1308_5626_gb300 import psp
    n, b = 50, 2
    Px = inputs.random_history(n, 4, seed=1)   # 4 columns < 2b+2 unknowns
    ref, sing = mrep.mrep(Px, 2 * Px, b)
    s = psp.Solver((n,), 2, [(2, 0, 1.0)], b, 8)
    out = torch.empty((n, 2 * b + 1), dtype=torch.float64, device=dev)
    ns = psp.psp_fit_band(s.handle, t64(Px.T, dev), t64(2 * Px.T, dev), out)
    assert ns == int(sing.sum()) == n - 2 * b
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=1e-12)
    s.close()
