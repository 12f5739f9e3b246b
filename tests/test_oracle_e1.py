"""The paper's mock test (Results section) on the oracle, CPU only.

A is the seeded random seven-diagonal, diagonally dominant matrix; u^n = (1, ..., n).  Two
steps of the step driver with d = 1: the first with N = I (plain restarted GMRES), the second
trying the tridiagonal N fitted to the first step's matvec history.  Pinned: both steps
reach the dense solution within the tolerance bound, the band storage round-trips, and the
fitted N of a system whose A is itself tridiagonal recovers A exactly (Algorithm 2's exact
recovery on the mock's own structure).
"""
import numpy as np
import pytest

from oracle import mrep
from oracle.explicit import MatrixOperator
from oracle.step import Stepper
from paper_1308_5626_gb300 import inputs


def test_band_storage_round_trip():
    A = inputs.mock_seven_diagonal(37, seed=1)
    band = inputs.dense_to_band(A, 3)
    B = np.zeros_like(A)
    for i in range(37):
        for p in range(7):
            j = i + p - 3
            if 0 <= j < 37:
                B[i, j] = band[i, p]
    np.testing.assert_array_equal(A, B)


@pytest.mark.parametrize("n", [20, 80, 150])
def test_mock_steps_reach_the_dense_solution(n):
    A = inputs.mock_seven_diagonal(n, seed=n)
    u = np.arange(1.0, n + 1.0)
    ref = np.linalg.solve(A, u)
    kappa = np.linalg.cond(A)
    st = Stepper(MatrixOperator(A), b=1, m=10)
    tol = 1e-10
    for step in range(2):
        x, info = st.step(u, 1.0, tol)
        assert info.converged
        assert np.linalg.norm(x - ref) <= kappa * 2 * tol * np.linalg.norm(ref), (step, info.iterations)


def test_tridiagonal_mock_is_recovered():
    rng = np.random.default_rng(9)
    n = 60
    A = np.diag(4.0 + rng.uniform(0, 1, n)) + np.diag(rng.uniform(-1, 1, n - 1), 1) + np.diag(rng.uniform(-1, 1, n - 1), -1)
    st = Stepper(MatrixOperator(A), b=1, m=10)
    st.step(np.arange(1.0, n + 1.0), 1.0, 1e-12)
    Px = np.stack(st.hist_x, axis=1)
    Py = np.stack(st.hist_y, axis=1)
    band, _ = mrep.mrep(Px, Py, 1, True)
    ref = inputs.dense_to_band(A, 1)
    # interior rows are A's rows; the first and last row keep only the diagonal (paper)
    np.testing.assert_allclose(band[1:-1], ref[1:-1], rtol=1e-8, atol=1e-8)


def _mock_golden():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "mock_test_setup.txt")
    out = {}
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].split()
            if line:
                out[line[0]] = line[1:]
    return out


def test_mock_inputs_follow_the_papers_setup():
    """The seeded inputs reproduce the setup the paper states (tests/golden/mock_test_setup.txt):
    its five sizes, a seven-diagonal diagonally dominant A, d = 1 (tridiagonal N), u^n = 1..n."""
    g = _mock_golden()
    assert tuple(int(v) for v in g["sizes"]) == inputs.MOCK_SIZES
    ndiag, d = int(g["diagonals"][0]), int(g["d"][0])
    for n in inputs.MOCK_SIZES[:3]:
        A = inputs.mock_seven_diagonal(n, seed=n)
        offs = {j - i for i, j in zip(*np.nonzero(A))}
        assert offs == set(range(-(ndiag // 2), ndiag // 2 + 1))
        off = np.abs(A).sum(axis=1) - np.abs(np.diag(A))
        assert np.all(np.abs(np.diag(A)) > off)            # strictly diagonally dominant
        # the fitted N has half-width d: tridiagonal storage (n, 2d + 1)
        rng = np.random.default_rng(n)
        Px = rng.standard_normal((n, 12))
        band, _ = mrep.mrep(Px, A @ Px, d)
        assert band.shape == (n, 2 * d + 1)
    assert g["rhs"] == ["arange", "1", "n"]
