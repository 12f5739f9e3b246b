"""Plain, slow FP64 CPU oracle for PSP-GMRES (Ghasemi & Taylor, arXiv:1308.5626).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import anything from this package.  The CUDA path never
calls it, and this package shares no code with the CUDA path: the only module both sides
use is ``paper_1308_5626_gb300.inputs`` (seeded input draws, no arithmetic of the method).

Modules, each following the passage it cites:

* ``fd``        central finite-difference weights for Eq. 1 (exact rationals).
* ``operator``  L and A = I - dt L of Eqs. 2-4, matrix-free (periodic shifts) and dense.
* ``exact``     the fixed result u^{n+1} = A^{-1} u^n: dense LU and the periodic
                Fourier-symbol solve 1 / (1 - dt lambda).
* ``banded``    the banded solve N^{-1} v (Thomas for d = 1, LAPACK band LU otherwise).
* ``gmres``     Algorithm 1 (PSP-GMRES with restarts and history capture).
* ``mrep``      Algorithm 2 (MREP: per-row least squares of P_y on P_x).
* ``step``      one implicit-Euler step driver with the progressive preconditioner.

Every function is pinned by ``tests/test_oracle_*.py`` to closed forms, textbook special
cases, brute force or invariants; none is marked "parity unpinned".
"""
