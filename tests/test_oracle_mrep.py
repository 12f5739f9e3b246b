"""Pins for oracle.mrep (Algorithm 2).

* Exact recovery: when A is banded within d and the history has full rank (m >= 2d+2),
  P_y = A P_x holds exactly, so every interior row of N equals A's row and the
  intercept vanishes; the boundary slope equals A(i, i) when that row is diagonal.
* Agreement with an independent least-squares routine (numpy lstsq, SVD-based) row by
  row on random data, with and without the intercept, and with scipy.stats.linregress
  for the boundary rows.
* Degenerate data (too few columns, repeated regressor rows) is flagged and gets the
  identity row.
"""
import numpy as np
import pytest
import scipy.stats

from oracle import banded, mrep
from paper_1308_5626_gb300 import inputs


@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("intercept", [True, False])
def test_exact_recovery_of_banded_A(d, intercept):
    n, m = 60, 3 * (2 * d + 2)
    A = banded.band_to_dense(inputs.random_band(n, d, seed=d), d)
    Px = inputs.random_history(n, m, seed=10 + d)
    Py = A @ Px
    band, sing = mrep.mrep(Px, Py, d, intercept)
    assert not sing.any()
    Aband = banded.dense_to_band(A, d)
    np.testing.assert_allclose(band[d:n - d], Aband[d:n - d], rtol=0, atol=1e-10 * np.abs(A).max())
    # boundary rows hold only the diagonal slope
    for i in list(range(d)) + list(range(n - d, n)):
        assert np.count_nonzero(band[i]) <= 1


def test_boundary_slope_of_diagonal_rows():
    n, d, m = 30, 2, 12
    diag = np.random.default_rng(3).uniform(1, 3, n)
    Px = inputs.random_history(n, m, seed=4)
    band, sing = mrep.mrep(Px, diag[:, None] * Px, d)
    np.testing.assert_allclose(band[:, d], diag, rtol=1e-12)
    np.testing.assert_allclose(np.delete(band, d, axis=1), 0.0, atol=1e-12)


@pytest.mark.parametrize("d", [1, 3])
@pytest.mark.parametrize("intercept", [True, False])
def test_matches_lstsq_on_random_data(d, intercept):
    n, m = 40, 25
    rng = np.random.default_rng(5 + d)
    Px = rng.standard_normal((n, m))
    Py = rng.standard_normal((n, m))
    band, sing = mrep.mrep(Px, Py, d, intercept)
    assert not sing.any()
    for i in range(d, n - d):
        rows = [np.ones(m)] if intercept else []
        rows += [Px[j] for j in range(i - d, i + d + 1)]
        X = np.stack(rows, axis=1)
        beta = np.linalg.lstsq(X, Py[i], rcond=None)[0]
        np.testing.assert_allclose(band[i], beta[1:] if intercept else beta, rtol=1e-9, atol=1e-12)
    for i in list(range(d)) + list(range(n - d, n)):
        if intercept:
            slope = scipy.stats.linregress(Px[i], Py[i]).slope
        else:
            slope = np.dot(Px[i], Py[i]) / np.dot(Px[i], Px[i])
        assert band[i, d] == pytest.approx(slope, rel=1e-10)


def test_degenerate_rows_are_flagged():
    n, d = 20, 1
    Px = inputs.random_history(n, 3, seed=1)            # 3 columns < 2d + 2 = 4 unknowns
    band, sing = mrep.mrep(Px, Px * 2.0, d)
    assert sing[d:n - d].all() and not sing[:d].any()
    np.testing.assert_array_equal(band[d:n - d], np.tile([0.0, 1.0, 0.0], (n - 2 * d, 1)))
    Px = inputs.random_history(n, 10, seed=2)
    Px[7] = Px[8]                                        # repeated regressor rows
    band, sing = mrep.mrep(Px, Px, d)
    assert sing[7] and sing[8] and not sing[6] and not sing[9]


def test_scatter_index_reading():
    """N*(j) multiplies P_x(i - d + j - 2, :): a pure shift A = S^{+1} is recovered as a
    1 on the first super-diagonal, not at the printed (out-of-band) column."""
    n, d, m = 25, 2, 12
    A = np.eye(n, k=1)
    Px = inputs.random_history(n, m, seed=7)
    band, _ = mrep.mrep(Px, A @ Px, d)
    np.testing.assert_allclose(band[d:n - d, d + 1], 1.0, atol=1e-12)
    np.testing.assert_allclose(np.delete(band[d:n - d], d + 1, axis=1), 0.0, atol=1e-12)
