"""Pins for oracle.banded: N^{-1} v against a dense LU and, for d = 1, the Thomas algorithm."""
import numpy as np
import pytest

from oracle import banded
from paper_1308_5626_gb300 import inputs


@pytest.mark.parametrize("b", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [9, 50, 257])
def test_solve_matches_dense(n, b):
    band = inputs.random_pd_part_band(n, b, seed=n + b)
    A = banded.band_to_dense(band, b)
    v = np.random.default_rng(n).standard_normal(n)
    np.testing.assert_allclose(banded.solve(band, b, v), np.linalg.solve(A, v), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(banded.solve(band, b, v, transpose=True), np.linalg.solve(A.T, v),
                               rtol=1e-10, atol=1e-12)


def test_band_round_trip_and_transpose():
    band = inputs.random_band(20, 3, seed=4)
    A = banded.band_to_dense(band, 3)
    np.testing.assert_array_equal(banded.dense_to_band(A, 3), band)
    np.testing.assert_array_equal(banded.band_to_dense(banded.transpose_band(band, 3), 3), A.T)


@pytest.mark.parametrize("n", [2, 3, 40, 333])
def test_thomas_equals_band_lu(n):
    band = inputs.random_band(n, 1, seed=n)
    v = np.random.default_rng(1).standard_normal(n)
    np.testing.assert_allclose(banded.thomas(band, v), banded.solve(band, 1, v), rtol=1e-12, atol=1e-13)
