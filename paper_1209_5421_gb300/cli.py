"""Solve a named synthetic workload once (or a few times) on the GPU and print the result.

  python -m paper_1209_5421_gb300.cli --workload quasi_uniform_1025 --prec fp32 --outer fgmres
  python -m paper_1209_5421_gb300.cli --batch 256 --prec fp32 --repeat 10

Workloads: see paper_1209_5421_gb300.meshes.WORKLOADS. Inputs are copied to the device first;
each repetition runs amg_setup + amg_solve + amg_free through the C ABI. With --batch N: the
first N systems of the batched workload (meshes.batch_workload) set up once by amg_batch_setup
and solved `repeat` times by amg_batch_solve (the first solve also times the launch shapes).
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
    ap.add_argument("--batch", type=int, default=0)
    a = ap.parse_args(argv)
    if a.batch > 0:
        return batch_main(a)
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


def batch_main(a) -> int:
    import numpy as np
    import torch

    from . import amg
    from .meshes import batch_workload

    probs = batch_workload(count=a.batch)
    cat = amg.concatenate([(p.rowptr, p.col, p.val, p.x, p.y) for p in probs], device="cuda")
    rhs = torch.as_tensor(np.concatenate([p.b for p in probs])).cuda()
    x = torch.empty_like(rhs)
    B = amg.Batch(concatenated=cat, cycle_prec=amg.FP32 if a.prec == "fp32" else amg.FP64)
    status = 0
    for _ in range(a.repeat):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, it, rr, st = B.solve(rhs, a.tol, x=x)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        print(f"batch of {a.batch} systems ({int(cat[0][-1])} unknowns), {a.prec} cycle: "
              f"{int(it.min())}-{int(it.max())} iterations, relres <= {rr.max():.3e}, "
              f"{1e3 * dt:.2f} ms, {B.moved_bytes() / 1e9:.1f} GB moved", flush=True)
        status = status or int((st != amg.OK).any())
    B.close()
    return status


if __name__ == "__main__":
    sys.exit(main())
