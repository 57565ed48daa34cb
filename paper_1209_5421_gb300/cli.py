"""Solve a named synthetic workload once (or a few times) on the GPU and print the result.

  python -m paper_1209_5421_gb300.cli --workload quasi_uniform_1025 --prec fp32 --outer fgmres

Workloads: see paper_1209_5421_gb300.meshes.WORKLOADS. Inputs are copied to the device first;
each repetition runs amg_setup + amg_solve + amg_free through the C ABI.
"""
from __future__ import annotations

import argparse
import sys
import time


def main(argv=None) -> int:
    import torch

    from . import amg
    from .meshes import WORKLOADS, workload

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="quasi_uniform_1025", choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--outer", default="fcg", choices=["fcg", "fgmres"])
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--repeat", type=int, default=1)
    a = ap.parse_args(argv)
    prob, aux = workload(a.workload)
    dev = lambda t: torch.as_tensor(t).cuda()  # noqa: E731
    A = [dev(t) for t in (prob.rowptr, prob.col, prob.val, prob.x, prob.y)]
    b = dev(prob.b)
    x = torch.empty_like(b)
    z = dev(prob.z) if getattr(prob, "z", None) is not None else None  # octree (3D)
    opts = dict(aux_level=aux, z=z, cycle_prec=amg.FP32 if a.prec == "fp32" else amg.FP64,
                outer=amg.OUTER_FGMRES if a.outer == "fgmres" else amg.OUTER_FCG)
    status = 0
    for _ in range(a.repeat):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = amg.Hierarchy(*A, **opts)
        _, it, rr, st = h.solve(b, a.tol, x=x)
        h.close()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        print(f"{a.workload}: {prob.n} unknowns, {a.prec} cycle, {a.outer} outer: "
              f"{it} iterations, relres {rr:.3e}, status {amg.status_string(st)}, "
              f"{1e3 * dt:.2f} ms", flush=True)
        status = status or (st != amg.OK)
    return int(status)


if __name__ == "__main__":
    sys.exit(main())
