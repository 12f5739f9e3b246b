"""Micro-benchmarks of single operations of the step, through the C ABI, on seeded synthetic
inputs of the 3D workload's operator (256^3 grid, 8th order, radius 5 in every direction,
rho(L) dt = 100; band half-width b = 3 for the preconditioner).

    python -m paper_1308_5626_gb300.kernel_bench stencil [--n3 256] [--fp64] [--reps 20]
    python -m paper_1308_5626_gb300.kernel_bench precond [--n3 256] [--fp64] [--reps 20]
    python -m paper_1308_5626_gb300.kernel_bench cycle [--n3 256] [--m 8] [--steps 2] [--fp64]

`stencil` times y = A x (psp_matvec), `precond` the banded solve y = N^{-1} v with a random
diagonally dominant band (psp_apply_precond), each as the mean and the minimum of --reps calls
bracketed by CUDA events on the handle's stream after 3 untimed calls.  `cycle` runs --steps
implicit steps of the workload with a restart length of --m (and a history of 2 (m + 1)
columns), so that a profiler can capture the in-cycle kernels (the stencil with its history
copy, the Gram-Schmidt passes, the restart residual) at the full grid with a few GB on the
device.  Each command prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import sys


def _timed(stream, call, reps):
    import torch
    for _ in range(3):
        call()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return sum(ts) / len(ts), min(ts)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("op", choices=["stencil", "precond", "cycle"])
    ap.add_argument("--n3", type=int, default=256, help="grid points per direction")
    ap.add_argument("--fp64", action="store_true", help="FP64 vectors (default: the mixed form's FP32)")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--m", type=int, default=8, help="restart length of `cycle`")
    ap.add_argument("--steps", type=int, default=2, help="implicit steps of `cycle`")
    a = ap.parse_args(argv)

    import torch

    from paper_1308_5626_gb300 import inputs, psp

    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    w = inputs.c3(a.n3, with_u0=(a.op == "cycle"))
    prec = psp.PSP_FP64 if a.fp64 else psp.PSP_MIXED
    dt_t = torch.float64 if a.fp64 else torch.float32
    es = 8 if a.fp64 else 4
    n = a.n3 ** 3
    m = a.m if a.op == "cycle" else 2
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        s = psp.Solver(w.shape, w.order, w.terms, w.b, m, precision=prec, stream=stream, onchip=0,
                       max_hist_cols=2 * (m + 1))
        dt = psp.workload_dt(w)
        line = {"op": a.op, "grid": [a.n3] * 3, "dtype": "f64" if a.fp64 else "f32"}
        if a.op == "stencil":
            g = torch.Generator(device=dev)
            g.manual_seed(7)
            x = torch.randn(n, dtype=dt_t, device=dev, generator=g)
            y = torch.empty_like(x)
            mean, best = _timed(stream, lambda: psp.psp_matvec(s.handle, x, y, dt), a.reps)
            line.update({"bytes": 2 * es * n})
        elif a.op == "precond":
            band = torch.tensor(inputs.random_band(n, w.b, seed=11), dtype=torch.float64, device=dev)
            psp.psp_set_band(s.handle, band)
            g = torch.Generator(device=dev)
            g.manual_seed(7)
            v = torch.randn(n, dtype=dt_t, device=dev, generator=g)
            y = torch.empty_like(v)
            mean, best = _timed(stream, lambda: psp.psp_apply_precond(s.handle, v, y), a.reps)
            line.update({"b": w.b, "bytes": 2 * es * n})
        else:
            u = torch.tensor(w.u0, dtype=torch.float64, device=dev)
            out = torch.empty_like(u)
            its = []
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(a.steps):
                _, info = s.step(u, dt, w.tol, out=out, allow_noconv=True)
                its.append(int(info.iters))
                u, out = out, u
            e1.record(stream)
            e1.synchronize()
            mean = best = e0.elapsed_time(e1) / a.steps
            line.update({"m": a.m, "steps": a.steps, "iters": its})
        s.close()
    line.update({"ms_mean": mean, "ms_min": best})
    if "bytes" in line:
        line["gbs_mean"] = line["bytes"] / (mean * 1e-3) / 1e9
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
