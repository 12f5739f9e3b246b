"""Pins of the oracle's cyclic band (oracle/banded.py, oracle/mrep.py with cyclic=True), CPU only.

The cyclic band reads band[i, p] as N(i, (i + p - d) mod n): the structure of a periodic 1D
stencil.  Pinned against what does not use the oracle's own assembly:

* storage: the wrapped entries land in the named corner cells of the dense matrix;
* solve: a circulant band (the same coefficients in every row) is diagonalised by the DFT,
  so N^{-1} v = ifft(fft(v) / lambda) with lambda_k = sum_s c_s exp(2 pi i k s / n), and
  N^{-T} v uses conj(lambda); a random cyclic band against a dense LU solve;
* fit: per-row numpy lstsq on the wrapped design rows (the first and last d rows
  included); a periodic 1D operator A whose stencil fits the band is recovered exactly in
  every row, while the paper's boundary rows leave the first and last d rows diagonal;
* step driver: with the cyclic fit, A N^{-1} = I, so every step after the first adopted
  candidate converges in one iteration and reaches the exact (Fourier) solution.
"""
import numpy as np
import pytest

from oracle import banded, exact, mrep
from oracle.operator import Operator
from oracle.step import Stepper
from paper_1308_5626_gb300 import inputs


def _cyclic_band(n, d, seed, dominant=True):
    rng = np.random.default_rng(seed)
    band = rng.uniform(-1.0, 1.0, (n, 2 * d + 1))
    if dominant:
        band[:, d] = 1.0 + np.abs(band).sum(axis=1)
    return band


def test_storage_corners():
    n, d = 9, 2
    band = np.arange(n * (2 * d + 1), dtype=float).reshape(n, 2 * d + 1) + 1.0
    A = banded.band_to_dense(band, d, cyclic=True)
    # row 0: columns -2, -1 wrap to n-2, n-1; row n-1: columns n, n+1 wrap to 0, 1
    assert A[0, n - 2] == band[0, 0] and A[0, n - 1] == band[0, 1] and A[0, 0] == band[0, 2]
    assert A[n - 1, 0] == band[n - 1, 3] and A[n - 1, 1] == band[n - 1, 4]
    assert np.count_nonzero(A) == n * (2 * d + 1)
    np.testing.assert_array_equal(banded.dense_to_band(A, d, cyclic=True), band)
    # the plain band drops exactly the wrapped cells
    assert np.count_nonzero(banded.band_to_dense(band, d)) == n * (2 * d + 1) - d * (d + 1)
    # transpose: N^T(i, j) = N(j, i) including the corners
    np.testing.assert_array_equal(banded.band_to_dense(banded.transpose_band(band, d, cyclic=True), d, cyclic=True),
                                  A.T)


@pytest.mark.parametrize("n,d", [(16, 1), (64, 2), (101, 3), (257, 4)])
def test_circulant_solve_by_dft(n, d):
    rng = np.random.default_rng(n)
    c = rng.uniform(-1.0, 1.0, 2 * d + 1)
    c[d] = 1.0 + np.abs(c).sum()
    band = np.tile(c, (n, 1))
    v = rng.standard_normal(n)
    s = np.arange(2 * d + 1) - d
    lam = np.array([np.sum(c * np.exp(2j * np.pi * k * s / n)) for k in range(n)])
    ref = np.real(np.fft.ifft(np.fft.fft(v) / lam))
    refT = np.real(np.fft.ifft(np.fft.fft(v) / np.conj(lam)))
    np.testing.assert_allclose(banded.solve(band, d, v, cyclic=True), ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    np.testing.assert_allclose(banded.solve(band, d, v, transpose=True, cyclic=True), refT, rtol=0,
                               atol=1e-13 * np.abs(refT).max())
    # the non-cyclic solve of the same storage is a different matrix
    assert np.abs(banded.solve(band, d, v) - ref).max() > 1e-6


@pytest.mark.parametrize("n,d", [(7, 3), (40, 2), (300, 4)])
def test_random_cyclic_solve_against_dense(n, d):
    band = _cyclic_band(n, d, seed=n + d)
    v = np.random.default_rng(1).standard_normal(n)
    A = banded.band_to_dense(band, d, cyclic=True)
    np.testing.assert_allclose(banded.solve(band, d, v, cyclic=True), np.linalg.solve(A, v), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("intercept", [True, False])
def test_cyclic_fit_rows_against_lstsq(intercept):
    n, d, M = 30, 2, 17
    rng = np.random.default_rng(7)
    Px = rng.standard_normal((n, M))
    Py = rng.standard_normal((n, M))
    band, sing = mrep.mrep(Px, Py, d, intercept, cyclic=True)
    assert not sing.any()
    for i in (0, 1, n // 2, n - 2, n - 1):
        rows = [(i + j - d) % n for j in range(2 * d + 1)]
        X = Px[rows].T
        if intercept:
            X = np.hstack([np.ones((M, 1)), X])
        beta = np.linalg.lstsq(X, Py[i], rcond=None)[0]
        np.testing.assert_allclose(band[i], beta[1:] if intercept else beta, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("order,terms", [(4, [(1, 0, 1.0), (2, 0, 0.01)]), (8, [(2, 0, 0.7), (4, 0, -1e-3)])])
def test_cyclic_fit_recovers_periodic_operator(order, terms):
    n = 64
    op = Operator((n,), order, terms)
    d = max(len(op.weights[(k, order)]) // 2 for k, _, _ in op.terms)   # stencil radius
    A = op.dense_A(0.3 * op.h[0])
    rng = np.random.default_rng(3)
    Px = rng.standard_normal((n, 2 * d + 6))
    Py = A @ Px
    band, sing = mrep.mrep(Px, Py, d, True, cyclic=True)
    assert not sing.any()
    np.testing.assert_allclose(banded.band_to_dense(band, d, cyclic=True), A, rtol=0, atol=1e-11)
    # the paper's boundary rows cannot represent the wrap: rows 0..d-1 keep only N(i, i)
    plain, _ = mrep.mrep(Px, Py, d, True)
    assert np.abs(banded.band_to_dense(plain, d) - A)[:d].max() > 1e-3


def test_cyclic_stepper_converges_in_one_iteration():
    w = inputs.c1(256)
    op = Operator(w.shape, w.order, w.terms)
    st = Stepper(op, w.b, w.m, cyclic=True)
    u = w.u0
    its = []
    for _ in range(4):
        u_next, info = st.step(u, w.dt, 1e-10)
        ref = exact.solve_fourier(op, u, w.dt)
        assert np.linalg.norm(u_next - ref) <= 1e-8 * np.linalg.norm(ref)
        its.append(info.iterations)
        u = u_next
    assert its[0] > 5          # N = I
    assert all(k == 1 for k in its[1:]), its
