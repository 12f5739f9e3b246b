"""Helpers shared by the GPU parity tests (imported only by tests marked gpu)."""
import numpy as np


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def torch_dev():
    import torch
    from paper_1308_5626_gb300 import build
    build.build()
    return torch.device("cuda:0")


def t64(a, dev):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


def t32(a, dev):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)


def rel_max(a, b):
    """Element-wise relative difference max|a - b| / max|b| (catches a localised error that
    a 2-norm dilutes)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def inv_inf_norm(op, dt):
    """||A^{-1}||_inf of the circulant A = I - dt L on the operator's periodic grid: every row
    of A^{-1} is a cyclic shift of every other, so its absolute row sum is the absolute sum
    of the column A^{-1} e_0 (the oracle's Fourier solve of a unit impulse)."""
    from oracle import exact
    e0 = np.zeros(op.n)
    e0[0] = 1.0
    return float(np.abs(exact.solve_fourier(op, e0, dt)).sum())


def elementwise_bound(inv_inf, tol, u_n, ref):
    """Bound on max|x - x*| / max|x*| for an x whose residual ||u_n - A x||_2 <= tol ||u_n||_2:
    x - x* = A^{-1} r, so max|x - x*| <= ||A^{-1}||_inf max|r| <= ||A^{-1}||_inf tol ||u_n||_2.
    Doubled for the rounding of the exact reference."""
    return 2.0 * inv_inf * tol * float(np.linalg.norm(u_n)) / float(np.abs(ref).max())
