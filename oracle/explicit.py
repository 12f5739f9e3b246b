"""An explicit matrix as the operator of the step driver: the paper's mock test (Results
section), where A of Eq. 4 is a given random seven-diagonal matrix and u^n = (1, ..., n).

Test infrastructure: only the tests and the bench's CPU legs use this module.  The step
driver (``oracle.step.Stepper``) calls ``apply_A(x, dt)``; here dt plays no role (A is
given, not I - dt L).
"""
from __future__ import annotations

import numpy as np


class MatrixOperator:
    def __init__(self, A: np.ndarray) -> None:
        self.A = np.asarray(A, dtype=np.float64)
        self.shape = (self.A.shape[0],)

    @property
    def n(self) -> int:
        return self.A.shape[0]

    def apply_A(self, x: np.ndarray, dt: float = 0.0) -> np.ndarray:
        return self.A @ np.asarray(x, dtype=np.float64)
