"""Differentiable implicit-Euler step on top of the C ABI.

`ImplicitStep.apply(u_n, dt, alpha, problem)` returns u^{n+1} = A^{-1} u^n (Eq. 4) by
`psp_step` on a forward handle.  Its backward solves the adjoint system
A^T lambda = g (g = dLoss/du^{n+1}) by the same matrix-free restarted GMRES on an adjoint
handle (`psp_opts.adjoint = 1`: every stencil mirrored), preconditioned by N^T of the
forward handle's adopted N, and returns

    dLoss/du^n = lambda,  dLoss/d(dt) = lambda . L u^{n+1},  dLoss/d(alpha_t) = dt lambda . D_t u^{n+1}

(the derivative of A u^{n+1} = u^n) from one `psp_adjoint_grads` call on the forward
handle, and N^T reaches the adjoint handle through `psp_set_band_from(adj, fwd, 1)`.  All
arithmetic of the step, the adjoint solve, the transposed band and the gradient dot products
runs in the library's kernels; this module only marshals arguments.

`rollout(..., checkpoint=True)` keeps only the input of every step and recomputes the step
during the backward pass (torch.utils.checkpoint), so a long rollout stores one vector per
step instead of the autograd graph's intermediates.
"""
from __future__ import annotations

from collections import OrderedDict
from typing import Sequence, Tuple

from . import psp


class Problem:
    """A family of implicit steps: grid, stencil order, the (k, dir) of each term, band
    half-width b, restart m, precision and relative tolerance.  Holds one forward and one
    adjoint handle per coefficient vector (least recently used first out)."""

    def __init__(self, shape: Sequence[int], order: int, kdirs: Sequence[Tuple[int, int]], b: int, m: int,
                 precision: int = psp.PSP_FP64, tol: float = 1e-12, max_cached: int = 4, stream=None):
        self.shape = tuple(int(s) for s in shape)
        self.order = int(order)
        self.kdirs = [(int(k), int(d)) for k, d in kdirs]
        self.b, self.m = int(b), int(m)
        self.precision = int(precision)
        self.tol = float(tol)
        self.max_cached = int(max_cached)
        self.stream = stream
        self._cache: "OrderedDict[tuple, dict]" = OrderedDict()

    def _terms(self, alphas):
        return [(k, d, float(a)) for (k, d), a in zip(self.kdirs, alphas)]

    def entry(self, alphas: tuple) -> dict:
        e = self._cache.get(alphas)
        if e is None:
            terms = self._terms(alphas)
            e = {
                "fwd": psp.Solver(self.shape, self.order, terms, self.b, self.m, precision=self.precision,
                                  stream=self.stream),
                "adj": psp.Solver(self.shape, self.order, terms, self.b, self.m, precision=self.precision,
                                  adjoint=1, stream=self.stream),
                "nt_stale": False,   # the forward adopted a new N since N^T was handed over
            }
            self._cache[alphas] = e
            while len(self._cache) > self.max_cached:
                _, old = self._cache.popitem(last=False)
                old["fwd"].close()
                old["adj"].close()
        else:
            self._cache.move_to_end(alphas)
        return e

    def close(self):
        for e in self._cache.values():
            e["fwd"].close()
            e["adj"].close()
        self._cache.clear()


class ImplicitStep:
    """torch.autograd.Function wrapper, built lazily so that importing the package does not
    import torch."""

    _fn = None

    @classmethod
    def apply(cls, u_n, dt, alpha, problem: Problem):
        if cls._fn is None:
            cls._fn = _make_function()
        return cls._fn.apply(u_n, dt, alpha, problem)


def _make_function():
    import torch

    class _Step(torch.autograd.Function):
        @staticmethod
        def forward(ctx, u_n, dt, alpha, problem):
            alphas = tuple(float(v) for v in alpha.detach().reshape(-1).cpu().tolist())
            e = problem.entry(alphas)
            u1, info = e["fwd"].step(u_n.detach().to(torch.float64).contiguous(), float(dt), problem.tol)
            if info.flags & psp.PSP_FLAG_CANDIDATE_ACCEPTED:
                e["nt_stale"] = True
            ctx.problem = problem
            ctx.alphas = alphas
            ctx.dt = float(dt)
            ctx.dt_like = dt
            ctx.alpha_like = alpha
            ctx.save_for_backward(u1)
            return u1

        @staticmethod
        def backward(ctx, g):
            (u1,) = ctx.saved_tensors
            problem = ctx.problem
            e = problem.entry(ctx.alphas)
            fwd, adj = e["fwd"], e["adj"]
            if e["nt_stale"]:
                psp.psp_set_band_from(adj.handle, fwd.handle, 1)
                e["nt_stale"] = False
            lam, _ = adj.step(g.detach().to(torch.float64).contiguous(), ctx.dt, problem.tol)
            grads = psp.psp_adjoint_grads(fwd.handle, lam, u1, ctx.dt, len(problem.kdirs))
            ddt = torch.tensor(grads[0], dtype=ctx.dt_like.dtype, device=ctx.dt_like.device).reshape(
                ctx.dt_like.shape) if torch.is_tensor(ctx.dt_like) else None
            dalpha = torch.tensor(grads[1:], dtype=ctx.alpha_like.dtype, device=ctx.alpha_like.device).reshape(
                ctx.alpha_like.shape)
            return lam, ddt, dalpha, None

    return _Step


def rollout(u0, dt, alpha, problem: Problem, steps: int, checkpoint: bool = False):
    """u^steps after `steps` implicit steps; differentiable in u0, dt and alpha."""
    import torch
    u = u0
    for _ in range(steps):
        if checkpoint:
            from torch.utils.checkpoint import checkpoint as ckpt
            u = ckpt(lambda x, d, a: ImplicitStep.apply(x, d, a, problem), u, dt, alpha, use_reentrant=False)
        else:
            u = ImplicitStep.apply(u, dt, alpha, problem)
    return u
