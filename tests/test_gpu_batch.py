"""GPU parity of the batched step (psp_step_batch): independent instances of the batched
workload's recipe, stepped together by a pool of host threads.

* Every instance's result equals the exact solve of its own step (Fourier, oracle) within
  kappa * 2 tol (mixed form, tol 1e-8 as the batched configuration asks).
* The batch is deterministic and free of cross-instance interference: each instance equals
  the same instance stepped alone by psp_step on a twin handle, to 1e-13.
* Handles that share one stream still run concurrently and in order: the batch reads inputs
  that were written on that stream behind a long kernel, without a host synchronisation.
* FP64 and mixed handles in one batch: the batched on-chip launches take one precision, the
  host threads step the rest, each still equal to its single step.
* A handle listed twice is refused (PSP_ERR_ARG) before any instance is stepped.
"""
import numpy as np
import pytest

from gpu_common import rel, t64, torch_dev
from oracle import exact
from oracle.operator import Operator
from paper_1308_5626_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return torch_dev()


@pytest.mark.parametrize("onchip", [0, 1], ids=["graphs", "onchip"])
def test_batch_matches_exact_and_single(dev, onchip):
    """onchip = 0: the instances' cycle graphs driven by host threads; onchip = 1: the
    persistent launches of the on-chip path (one CTA per system) run every instance's cycles.
    Either way every instance equals its exact solve within cond(A) 2 tol and the same
    instance stepped alone (the same arithmetic) to rounding."""
    import torch
    from paper_1308_5626_gb300 import psp
    ws = [inputs.c4_instance(i, e_range=(8, 12)) for i in range(12)]

    def make(w):
        s = torch.cuda.Stream(device=dev)
        return psp.Solver(w.shape, w.order, w.terms, w.b, w.m, precision=psp.PSP_MIXED, stream=s, onchip=onchip)

    batch = [make(w) for w in ws]
    twins = [make(w) for w in ws]
    us = [t64(w.u0, dev) for w in ws]
    outs = [torch.empty_like(u) for u in us]
    refs = [w.u0 for w in ws]
    tol = 1e-8
    for step in range(2):
        torch.cuda.synchronize()
        infos, secs, sts = psp.psp_step_batch([s.handle for s in batch], us, outs, [w.dt for w in ws], tol,
                                              nthreads=4)
        torch.cuda.synchronize()
        assert all(st == 0 for st in sts), sts
        assert all(t > 0.0 for t in secs)
        for i, w in enumerate(ws):
            op = Operator(w.shape, w.order, w.terms)
            ref = exact.solve_fourier(op, refs[i], w.dt)
            got = outs[i].cpu().numpy()
            assert rel(got, ref) <= exact.condition_number(op, w.dt) * 2 * tol, (step, i, rel(got, ref))
            single, info = twins[i].step(us[i], w.dt, tol)
            torch.cuda.synchronize()
            assert rel(got, single.cpu().numpy()) <= 1e-13, (step, i)
            assert info.iters == infos[i].iters, (step, i)
            refs[i] = got
        us, outs = outs, us
    for s in batch + twins:
        s.close()


def test_batch_on_one_shared_stream_follows_its_inputs(dev):
    """All handles on one stream (as when a framework hands out pooled streams): the inputs are
    written on that stream behind a ~25 ms spin kernel and the batch is called at once; every
    instance must step the new inputs (the batch's work follows the stream's), equal to its
    twin stepped alone, and later work on the stream must see the results."""
    import torch
    from paper_1308_5626_gb300 import psp
    ws = [inputs.c4_instance(i, e_range=(9, 12)) for i in range(8)]
    shared = torch.cuda.Stream(device=dev)
    batch = [psp.Solver(w.shape, w.order, w.terms, w.b, w.m, precision=psp.PSP_MIXED, stream=shared, onchip=0)
             for w in ws]
    twins = [psp.Solver(w.shape, w.order, w.terms, w.b, w.m, precision=psp.PSP_MIXED, onchip=0) for w in ws]
    src = [t64(w.u0, dev) for w in ws]
    us = [torch.zeros_like(u) for u in src]
    outs = [torch.empty_like(u) for u in src]
    tol = 1e-8
    torch.cuda.synchronize()
    with torch.cuda.stream(shared):
        torch.cuda._sleep(50_000_000)
        for u, x in zip(us, src):
            u.copy_(x)
    infos, secs, sts = psp.psp_step_batch([s.handle for s in batch], us, outs, [w.dt for w in ws], tol, nthreads=4)
    assert all(st == 0 for st in sts), sts
    with torch.cuda.stream(shared):
        copies = [o.clone() for o in outs]
    torch.cuda.synchronize()
    for i, w in enumerate(ws):
        single, info = twins[i].step(src[i], w.dt, tol)
        torch.cuda.synchronize()
        got = copies[i].cpu().numpy()
        assert rel(got, single.cpu().numpy()) <= 1e-13, i
        assert info.iters == infos[i].iters, i
        op = Operator(w.shape, w.order, w.terms)
        ref = exact.solve_fourier(op, w.u0, w.dt)
        assert rel(got, ref) <= exact.condition_number(op, w.dt) * 2 * tol, i
    for s in batch + twins:
        s.close()


def test_batch_of_mixed_precisions(dev):
    """FP64 and mixed handles in one batch, all asking for the on-chip path: the batched
    on-chip launches take the first handle's precision, and the host threads step the other
    handles one at a time on their own streams (psp_step, here each on its single-system
    on-chip launch), both at once.  Every instance equals its twin stepped alone by psp_step
    (to 1e-13; same iterations) and its exact solve (cond(A) 2 tol)."""
    import torch
    from paper_1308_5626_gb300 import psp
    ws = [inputs.c4_spec(k % 2 == 1, 10 + k % 3, 2 + 2 * (k % 4), 1 + k % 4, 4.0 + k, seed=900 + k) for k in range(6)]
    precs = [psp.PSP_FP64 if k % 2 == 0 else psp.PSP_MIXED for k in range(6)]

    def make(w, p):
        return psp.Solver(w.shape, w.order, w.terms, w.b, w.m, precision=p, stream=torch.cuda.Stream(device=dev),
                          onchip=1)

    batch = [make(w, p) for w, p in zip(ws, precs)]
    twins = [make(w, p) for w, p in zip(ws, precs)]
    us = [t64(w.u0, dev) for w in ws]
    outs = [torch.empty_like(u) for u in us]
    tol = 1e-8
    for step in range(2):
        torch.cuda.synchronize()
        infos, secs, sts = psp.psp_step_batch([s.handle for s in batch], us, outs, [w.dt for w in ws], tol,
                                              nthreads=3)
        torch.cuda.synchronize()
        assert all(st == 0 for st in sts), sts
        for i, w in enumerate(ws):
            got = outs[i].cpu().numpy()
            single, info = twins[i].step(us[i], w.dt, tol)
            torch.cuda.synchronize()
            assert rel(got, single.cpu().numpy()) <= 1e-13, (step, i)
            assert info.iters == infos[i].iters, (step, i)
            op = Operator(w.shape, w.order, w.terms)
            ref = exact.solve_fourier(op, us[i].cpu().numpy(), w.dt)
            assert rel(got, ref) <= exact.condition_number(op, w.dt) * 2 * tol, (step, i)
        us, outs = outs, us
    for s in batch + twins:
        s.close()


def test_batch_refuses_a_repeated_handle(dev):
    import torch
    from paper_1308_5626_gb300 import psp
    w = inputs.c4_instance(0)
    s = psp.Solver(w.shape, w.order, w.terms, w.b, w.m, precision=psp.PSP_MIXED)
    u = [t64(w.u0, dev), t64(w.u0, dev)]
    out = [torch.empty_like(u[0]), torch.empty_like(u[0])]
    with pytest.raises(RuntimeError):
        psp.psp_step_batch([s.handle, s.handle], u, out, [w.dt, w.dt], 1e-8, nthreads=2)
    s.close()


def test_batch_tuner_measures_every_candidate_and_keeps_exact_steps(dev):
    """psp_batch_tuner(1): the first calls run each size class on one candidate per call (cycle
    graphs, on-chip CTAs of 128 / 256 / 512), every step still equal to the exact solve within
    cond(A) 2 tol; afterwards every class has a decision and its instances keep it."""
    import torch
    from paper_1308_5626_gb300 import psp
    ws = [inputs.c4_spec(k % 2 == 1, 10 + 2 * (k % 3), 2 + 2 * (k % 4), 1 + k % 4, 5.0 + k, seed=700 + k)
          for k in range(8)]
    solvers = [psp.Solver(w.shape, w.order, w.terms, w.b, w.m, precision=psp.PSP_MIXED,
                          stream=torch.cuda.Stream(device=dev)) for w in ws]
    us = [t64(w.u0, dev) for w in ws]
    outs = [torch.empty_like(u) for u in us]
    refs = [w.u0 for w in ws]
    ops = [Operator(w.shape, w.order, w.terms) for w in ws]
    psp.psp_batch_tuner(1)
    try:
        for call in range(6):
            infos, secs, sts = psp.psp_step_batch([s.handle for s in solvers], us, outs, [w.dt for w in ws], 1e-8,
                                                  nthreads=4)
            torch.cuda.synchronize()
            for i, w in enumerate(ws):
                assert sts[i] == 0, (call, i)
                got = outs[i].cpu().numpy()
                ref = exact.solve_fourier(ops[i], refs[i], w.dt)
                assert rel(got, ref) <= exact.condition_number(ops[i], w.dt) * 2 * 1e-8, (call, i)
                refs[i] = got
            us, outs = outs, us
        table = psp.psp_batch_tuner(-1)
        assert {c["log2_n"] for c in table} == {10, 12, 14}
        for c in table:
            assert c["choice"] is not None, c
            assert all(v >= 1 for v in c["samples"].values()), c
    finally:
        psp.psp_batch_tuner(0)
        for s in solvers:
            s.close()
