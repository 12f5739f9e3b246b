"""GB300-native PSP-GMRES: one implicit-Euler step (I - dt*L) u^{n+1} = u^n solved by
matrix-free restarted GMRES with the progressive statistical banded preconditioner
(Ghasemi & Taylor, arXiv:1308.5626, Algorithms 1 and 2).

The compute path lives in ``libpsp.so`` (hand-written CUDA for sm_103a behind a C ABI
declared in ``include/psp.h``).  ``paper_1308_5626_gb300.psp`` is the thin ctypes
binding (``psp.Solver``: steps in FP64 or the mixed FP32/FP64 form, the explicit banded
operator of the paper's mock test, the cyclic band for periodic 1D grids, the BiCGSTAB
solver option, BDF2 / SDIRK2 steps, batched stepping of many handles);
``paper_1308_5626_gb300.autograd`` makes the step differentiable (adjoint solve);
``paper_1308_5626_gb300.inputs`` holds the seeded synthetic workloads.

Importing this package loads nothing: the shared library is opened on first use of
``paper_1308_5626_gb300.psp``.
"""

__all__ = ["inputs", "psp", "build", "autograd"]
