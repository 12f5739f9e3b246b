"""Pins of the oracle's integrators (oracle/integrators.py), CPU only.

* On a single Fourier mode (an eigenvector of L with eigenvalue lambda, z = dt lambda) the
  SDIRK2 step multiplies by the method's closed-form stability function
  R(z) = (1 + (1 - 2 gamma) z) / (1 - gamma z)^2, and BDF2 by the root recurrence
  u^{n+1} = (4 u^n - u^{n-1}) / (3 - 2 z); R(z) -> 0 as z -> -inf (L-stability).
* Temporal order: against the exact exp(lambda t) on a damped, advected mode, halving dt
  divides the error by ~4 for BDF2 and SDIRK2 and by ~2 for implicit Euler.
"""
import math

import numpy as np
import pytest

from oracle import integrators
from oracle.operator import Operator


def _mode(op, k):
    n = op.shape[0]
    x = np.arange(n)
    return np.exp(2j * np.pi * k * x / n)


def _lambda(op, k):
    return op.symbol_1d(0)[k]


def _solve_complex(op, v, dt):
    """Fourier solve that keeps complex data (the oracle's step maps a real vector)."""
    amp = 1.0 / (1.0 - dt * op.symbol())
    return np.fft.ifft(np.fft.fft(v) * amp)


def _apply_L_complex(op, v):
    return op.apply_L(v.real) + 1j * op.apply_L(v.imag)


class _Cop:
    """The operator with a complex apply_L, for driving the oracle integrators on one mode."""

    def __init__(self, op):
        self.op = op

    def apply_L(self, v):
        return _apply_L_complex(self.op, v)


def test_sdirk2_stability_function():
    op = Operator((64,), 4, [(1, 0, 1.0), (2, 0, 0.05)])
    g = integrators.GAMMA
    assert abs(g - (1 - 1 / math.sqrt(2))) < 1e-16
    for k in (1, 5, 20):
        v = _mode(op, k)
        lam = _lambda(op, k)
        for dt in (0.01, 0.3, 5.0):
            z = dt * lam
            R = (1 + (1 - 2 * g) * z) / (1 - g * z) ** 2
            got = integrators.sdirk2_step(_Cop(op), v, dt, solve=lambda o, w, d: _solve_complex(op, w, d))
            np.testing.assert_allclose(got, R * v, rtol=1e-12, atol=1e-12)
    # L-stability: the stiff limit is damped to zero
    z = -1e8
    assert abs((1 + (1 - 2 * g) * z) / (1 - g * z) ** 2) < 1e-7


def test_bdf2_recurrence():
    op = Operator((48,), 6, [(2, 0, 0.3), (1, 0, -0.7)])
    for k in (2, 11):
        v = _mode(op, k)
        lam = _lambda(op, k)
        dt = 0.2
        z = dt * lam
        u_nm1, u_n = v, 0.8 * v
        got = integrators.bdf2_step(op, u_nm1, u_n, dt, solve=lambda o, w, d: _solve_complex(op, w, d))
        np.testing.assert_allclose(got, (4 * 0.8 - 1) / (3 - 2 * z) * v, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(integrators.bdf2_rhs(np.array([3.0]), np.array([6.0])), [2.0])


@pytest.mark.parametrize("method,order", [("euler", 1), ("bdf2", 2), ("sdirk2", 2)])
def test_temporal_order(method, order):
    op = Operator((32,), 8, [(2, 0, 0.2), (1, 0, 1.0)])
    k = 2
    lam = _lambda(op, k)
    v = _mode(op, k)
    T = 1.0
    errs = []
    for steps in (40, 80, 160):
        dt = T / steps
        us = [v]
        for s in range(steps):
            if method == "euler" or (method == "bdf2" and s == 0):
                if method == "bdf2":
                    # start BDF2 with the exact value so that the start-up step does not
                    # limit the order
                    us.append(np.exp(lam * dt) * v)
                else:
                    us.append(_solve_complex(op, us[-1], dt))
            elif method == "bdf2":
                us.append(integrators.bdf2_step(op, us[-2], us[-1], dt, solve=lambda o, w, d: _solve_complex(op, w, d)))
            else:
                us.append(integrators.sdirk2_step(_Cop(op), us[-1], dt, solve=lambda o, w, d: _solve_complex(op, w, d)))
        errs.append(np.abs(us[-1] - np.exp(lam * T) * v).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    for r in rates:
        assert abs(r - order) < 0.15, (method, rates)


def test_rollout_real_vectors():
    op = Operator((40,), 4, [(2, 0, 0.1)])
    u0 = np.random.default_rng(0).standard_normal(40)
    for m in ("euler", "bdf2", "sdirk2"):
        us = integrators.rollout(op, u0, 0.05, 3, m)
        assert len(us) == 4 and all(np.isrealobj(u) for u in us)
    # diffusion only: every method damps the energy
    for m in ("bdf2", "sdirk2"):
        us = integrators.rollout(op, u0, 0.05, 5, m)
        assert np.linalg.norm(us[-1]) < np.linalg.norm(u0)
