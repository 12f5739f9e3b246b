"""Run the oracle's implicit-Euler time series on a workload and record, per step, the
Arnoldi iterations, restart cycles and preconditioner adoption, with the wall time of the
oracle on this machine.  Writes JSON to stdout (or --out).

Used to state how many iterations one implicit step of a workload takes when the
benchmark times the oracle on a bounded sample (a few Arnoldi iterations) and scales it
to implicit steps per second.  Calls nothing outside oracle/ and the seeded inputs.

    python -m oracle.record_iterations --workload c2 --steps 10 --out oracle/c2_series.json
    python -m oracle.record_iterations --workload c3 --first-step-only --out oracle/c3_series.json

``--first-step-only`` records the first step alone, as Algorithm 1 runs it there (N = I,
X_0 = B = u^0), without the Algorithm 2 fit that would follow it: on the 256^3 workload a
step takes the oracle minutes and the fit's stacked history tens of GB of host memory.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import gmres  # noqa: E402
from oracle.operator import Operator  # noqa: E402
from oracle.step import Stepper  # noqa: E402
from paper_1308_5626_gb300 import inputs  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--out", default=None)
    ap.add_argument("--first-step-only", action="store_true")
    a = ap.parse_args()
    w = inputs.WORKLOADS[a.workload]()
    op = Operator(w.shape, w.order, w.terms)
    dt = w.dt if w.dt is not None else w.with_dt(op.spectral_radius())
    if a.first_step_only:
        import numpy as np
        t0 = time.perf_counter()
        res = gmres.pspgmres(lambda x: op.apply_A(x, dt), w.u0, None, w.tol * float(np.linalg.norm(w.u0)), w.m,
                             w.u0, 200)
        row = {"step": 0, "iterations": res.iterations, "cycles": res.cycles, "converged": bool(res.converged),
               "tried": False, "accepted": False, "seconds": time.perf_counter() - t0}
        out = {"workload": w.name, "dt": dt, "tol": w.tol, "m": w.m, "b": w.b, "steps": [row],
               "first_step_only": True, "mean_iterations": float(res.iterations), "mean_cycles": float(res.cycles)}
        txt = json.dumps(out, indent=1)
        if a.out:
            with open(a.out, "w") as fh:
                fh.write(txt + "\n")
        else:
            print(txt)
        return
    st = Stepper(op, b=w.b, m=w.m)
    u = w.u0
    rows = []
    for s in range(a.steps):
        t0 = time.perf_counter()
        u, info = st.step(u, dt, w.tol)
        rows.append({"step": s, "iterations": info.iterations, "cycles": info.cycles,
                     "converged": bool(info.converged), "tried": bool(info.tried_candidate),
                     "accepted": bool(info.accepted), "seconds": time.perf_counter() - t0})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    out = {"workload": w.name, "dt": dt, "tol": w.tol, "m": w.m, "b": w.b, "steps": rows,
           "mean_iterations": sum(r["iterations"] for r in rows) / len(rows),
           "mean_cycles": sum(r["cycles"] for r in rows) / len(rows)}
    txt = json.dumps(out, indent=1)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(txt + "\n")
    else:
        print(txt)


if __name__ == "__main__":
    main()
