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
