"""Benchmark: solves/s (and p50/p99 latency) of the auxiliary-grid AMG on one GB300.

One step = one whole pass of the method over one synthetic system: amg_setup (binning,
aggregation, Galerkin operators, colouring, coarsest factorisation) + amg_solve to a 1e-8
relative residual + amg_free. Inputs (CSR, coordinates, rhs) are resident in HBM when the
timed region starts; L2 is flushed (a 256 MiB write) before every timed step, outside the
step's CUDA events.

Default workload: 1025 x 1025 jittered P1 Poisson (1,046,529 unknowns), auxiliary grid
1024 x 1024, FP32 AMLI-cycle inside FP64 restarted flexible GMRES, tol 1e-8. The plain FP64
method (FP64 cycle, flexible-CG outer) is timed on the same workload and reported beside it.

  value : solves/s of the whole job (N ranks x steps / max-over-ranks time)
  e2e   : the same, through the C ABI with pinned HOST buffers (copies inside the step)
  roofline : the dominant kernel's algorithmic bytes / its CUDA-event duration, from a
             profiling pass of the same workload and launch configuration
  cpu_baseline : the FP64 CPU oracle on this machine's host cores

--impl reference times the FP64 CPU oracle (the only reference implementation of this path)
on the same workload. Multi-GPU: independent replicas per rank (the method is one problem
per GPU; ranks do not exchange data), scaling "weak".
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "solves/s at 1e-8 rel. residual (setup+solve)"
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="quasi_uniform_1025")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--prec", default="fp32", choices=["fp64", "fp32"])
    ap.add_argument("--outer", default="fgmres", choices=["fcg", "fgmres"])
    ap.add_argument("--no-fp64-line", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-profile", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--no-graded", action="store_true")
    ap.add_argument("--batch-systems", type=int, default=256)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-octree", action="store_true")
    ap.add_argument("--octree-n", type=int, default=129)
    ap.add_argument("--serve-rates", default="10,50,100,200,500,1000,2000")
    ap.add_argument("--serve-requests", type=int, default=48)
    # systems above this many unknowns take the large lane (the grid-wide solver, alone on
    # the GPU); smaller ones share the batch lane, one CTA each
    ap.add_argument("--serve-large", type=int, default=50_000)
    return ap.parse_args()


# ---------------------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# the sources the measured solve kernels (the persistent cycle kernel and the batch kernel)
# are compiled from: the DRAM counters recorded under profiles/ hold while these are unchanged
KERNEL_SOURCES = ("amg_internal.cuh", "batch.cu", "batch_graded.cu", "batch_kernel.cuh",
                  "cycle_ops.cuh", "solve.cu")


def kernel_source_hash():
    import hashlib

    hsh = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1209_5421_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            hsh.update(fh.read())
    return hsh.hexdigest()[:16]


def recorded_traffic(workload, prec):
    """DRAM bytes per launch of the cycle kernel (or of the batch kernel: one launch is a
    whole batch solve) from the committed ncu summary, if it was taken on the current kernel
    sources (else None)."""
    p = os.path.join(ROOT, "profiles", "cycle_traffic.json")
    try:
        with open(p) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    key = f"{workload}:{prec}"
    ent = rec.get(key)
    if not ent or ent.get("source_hash") != kernel_source_hash():
        return None
    return ent.get("dram_bytes_per_launch")


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------------------
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl"
        try:
            import torch

            if not torch.cuda.is_available():
                backend = "gloo"
        except ImportError:
            backend = "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, v: float) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_baseline(prob, aux, tol, budget_s=30.0):
    """The FP64 CPU oracle, as it stands, on this machine's host cores (one thread)."""
    from oracle import oracle

    oracle.build()
    t0 = time.perf_counter()
    O = oracle.Hierarchy.from_problem(prob, aux_level=aux)
    t1 = time.perf_counter()
    x, it, rr, st = O.solve(prob.b, tol)
    t2 = time.perf_counter()
    return {"setup_s": t1 - t0, "solve_s": t2 - t1, "iters": it, "relres": rr, "status": st,
            "x": x}


def rel_err(x, xo):
    """||x - x_oracle|| / ||x_oracle|| (the error against the FP64 oracle's solution)."""
    return float(np.linalg.norm(x - xo) / np.linalg.norm(xo))


# ---------------------------------------------------------------------------------------
def run_reference(args, world, rank):
    """Reference arm: the FP64 CPU oracle on the host cores, same workload and metric."""
    if rank != 0:
        return 0
    from oracle import oracle
    from paper_1209_5421_gb300.meshes import workload

    oracle.build()
    prob, aux = workload(args.workload)
    times = []
    its = None
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        O = oracle.Hierarchy.from_problem(prob, aux_level=aux)
        x, its, rr, st = O.solve(prob.b, args.tol)
        del O
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
        if sum(times) > 150.0 and len(times) >= 1:  # bounded: a few minutes at most
            break
    total = sum(times)
    value = len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": len(times), "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "unknowns": prob.n, "nnz": prob.nnz,
                   "aux_level": aux, "tol": args.tol, "iters": its},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": f"{len(times)} full oracle setup+solve(s) of {args.workload}"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args, world, flush, dev, stream):
    """The batched form: `batch_systems` independent jittered P1 Poisson systems of uneven
    sizes (n x n nodes, n log-uniform in [45, 450]) solved together by one persistent kernel
    (FP32 cycle, FP64 flexible-CG outer, tol as the headline), hierarchies resident. Beside
    it: the plain FP64 method (single-system solver, FP64 cycle) on a sample of the same
    systems solved one after another, and the batch's own FP64-cycle form."""
    import torch

    from paper_1209_5421_gb300 import amg
    from paper_1209_5421_gb300.meshes import batch_workload

    from oracle import oracle

    probs = batch_workload(count=args.batch_systems)
    peak_gbs, _ = measured_peak_hbm()
    off = np.concatenate([[0], np.cumsum([p.n for p in probs])])
    by_size = sorted(range(len(probs)), key=lambda k: probs[k].n)
    err_sample = sorted(set(by_size[::64] + [by_size[-1]]))
    oracle_x = {}
    oracle.build()
    rhs = torch.as_tensor(np.concatenate([p.b for p in probs])).to(dev)
    x = torch.empty_like(rhs)
    # the block-diagonal CSR on the device (host-side concatenation in the binding, timed
    # apart); the setup time is the library's batched setup from there
    t0 = time.perf_counter()
    cat = amg.concatenate([(p.rowptr, p.col, p.val, p.x, p.y) for p in probs], device=dev)
    torch.cuda.synchronize()
    concat_s = time.perf_counter() - t0
    res = {}
    for name, prec in (("fp32", amg.FP32), ("fp64", amg.FP64)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B = amg.Batch(concatenated=cat, cycle_prec=prec)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        for _ in range(max(3, args.warmup)):  # the first solve also picks the launch shape
            flush.fill_(1.0)
            B.solve(rhs, args.tol, x=x)
        lat, its, rrs, sts, sys_lat = [], None, None, None, []
        barrier(world)
        for k in range(args.steps):
            flush.fill_(float(k))
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            _, its, rrs, sts = B.solve(rhs, args.tol, x=x)
            ev1.record(stream)
            torch.cuda.synchronize()
            lat.append(ev0.elapsed_time(ev1))
            sys_lat.extend((B.timeline()[1] / 1e6).tolist())
        barrier(world)
        t = max_over_ranks(world, sum(lat))
        info = B.info()
        team = B.teams()
        moved = B.moved_bytes()  # algorithmic bytes of one batch solve (the last one)
        B.close()
        # error against the FP64 oracle's solution, per result, on a sample of the systems
        # (every 64th in size order, the largest included)
        xh = x.cpu().numpy()
        errs = {}
        for k in err_sample:
            if k not in oracle_x:
                O = oracle.Hierarchy.from_problem(probs[k])
                oracle_x[k] = O.solve(probs[k].b, args.tol)[0]
            errs[int(probs[k].n)] = rel_err(xh[off[k]:off[k + 1]], oracle_x[k])
        if not (sts == amg.OK).all():
            raise RuntimeError(f"batched {name}: statuses {sorted(set(sts.tolist()))}")
        res[name] = {
            "value": round(world * len(probs) * args.steps / (t / 1e3), 2), "unit": "solves/s",
            "ms_per_batch": round(t / args.steps, 3),
            "setup_ms": round(1e3 * setup_s, 1),
            "host_concat_ms": round(1e3 * concat_s, 1),
            "with_setup": round(len(probs) / (setup_s + t / args.steps / 1e3), 2),
            "system_latency_ms": {"p50": round(float(np.percentile(sys_lat, 50)), 3),
                                  "p99": round(float(np.percentile(sys_lat, 99)), 3)},
            "iters": [int(its.min()), int(its.max())], "relres_max": float(rrs.max()),
            "err_vs_oracle": {"by_unknowns": errs, "max": max(errs.values())},
            "launch_shape": {"threads": info["threads"], "ctas": info["ctas"],
                             "tuned_ms": [round(v, 2) for v in info["tuned_ms"]]},
            "teams": {"systems": int((team > 1).sum()), "ctas": int(team[team > 1].sum()),
                      "largest": int(team.max())},
            "device_bytes": info["bytes"],
            # the batched kernel's roofline: algorithmic bytes of the whole batch solve (every
            # system's cycles and outer steps) over the batch's time; ncu counts about as
            # much DRAM traffic (the recorded `traffic`)
            "roofline": {"bound": "hbm", "kernel": "k_batch (whole batch solve)",
                         "achieved": round(moved / (t / args.steps / 1e3) / 1e9, 1),
                         "peak": peak_gbs, "unit": "GB/s",
                         "frac": round(moved / (t / args.steps / 1e3) / 1e9 / peak_gbs, 4),
                         "bytes_per_solve": moved,
                         # DRAM bytes of one batch-kernel launch (one whole batch solve) from
                         # the committed ncu summary, if taken on the current kernel sources
                         "traffic": recorded_traffic(f"batch_{len(probs)}", name)},
        }
    # the plain FP64 method, one system at a time (every 16th system, hierarchies resident)
    sample = probs[::16]
    hs = [amg.Hierarchy.from_problem(p, cycle_prec=amg.FP64) for p in sample]
    bs = [torch.as_tensor(p.b).to(dev) for p in sample]
    xs = [torch.empty_like(b) for b in bs]
    for h, b, xx in zip(hs, bs, xs):
        h.solve(b, args.tol, x=xx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for h, b, xx in zip(hs, bs, xs):
        _, _, _, st = h.solve(b, args.tol, x=xx)
        if st != amg.OK:
            raise RuntimeError(f"single-system FP64 solve failed: {st}")
    torch.cuda.synchronize()
    seq = time.perf_counter() - t0
    for h in hs:
        h.close()
    return {
        "workload": f"{len(probs)} jittered P1 Poisson systems, n x n nodes, n log-uniform in "
                    f"[45, 450] ({sum(p.n for p in probs)} unknowns)",
        "method": "FP32 AMLI-cycle, FP64 flexible-CG outer, one CTA (or a team of CTAs for "
                  "the largest systems) per system",
        **res.pop("fp32"),
        "fp64_cycle_batched": res["fp64"],
        "fp64_plain_sequential": {
            "value": round(len(sample) / seq, 2), "unit": "solves/s",
            "sample": f"every 16th system ({len(sample)} systems, "
                      f"{sum(p.n for p in sample)} unknowns), single-system FP64 solver, "
                      "one after another"},
    }


def run_octree(args, world, flush, dev, stream):
    """The octree (3D) variant: P1 Poisson on the unit cube, an octree_n^3-node Kuhn
    tetrahedral grid with jittered interior nodes ((octree_n - 2)^3 unknowns), setup + solve
    per step like the headline (FP32 AMLI-cycle with FGMRES(30), and the plain FP64 method)."""
    import torch

    from paper_1209_5421_gb300 import amg
    from paper_1209_5421_gb300.meshes import p1_poisson_3d

    prob = p1_poisson_3d(args.octree_n, seed=0)  # (cube_129 in meshes.WORKLOADS at 129)
    td = lambda a: torch.as_tensor(a).to(dev)  # noqa: E731
    A = [td(a) for a in (prob.rowptr, prob.col, prob.val, prob.x, prob.y)]
    z = td(prob.z)
    b = td(prob.b)
    x = torch.empty_like(b)
    out = {"workload": f"3D jittered P1 Poisson, {args.octree_n}^3-node Kuhn tetrahedral grid",
           "unknowns": prob.n, "nnz": prob.nnz}
    steps = max(1, min(args.steps, 5))
    for name, o in (("fp32_fgmres", dict(cycle_prec=amg.FP32, outer=amg.OUTER_FGMRES)),
                    ("fp64_fcg", dict(cycle_prec=amg.FP64, outer=amg.OUTER_FCG))):
        def step():
            h = amg.Hierarchy(*A, z=z, **o)
            _, it, rr, st = h.solve(b, args.tol, x=x)
            nlev = h.nlev
            h.close()
            if st != amg.OK:
                raise RuntimeError(f"octree {name}: status {st}, relres {rr}")
            return it, nlev

        for _ in range(max(1, args.warmup)):
            flush.fill_(1.0)
            step()
        torch.cuda.synchronize()
        barrier(world)
        lat = []
        for k in range(steps):
            flush.fill_(float(k))
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            it, nlev = step()
            ev1.record(stream)
            torch.cuda.synchronize()
            lat.append(ev0.elapsed_time(ev1))
        barrier(world)
        t = max_over_ranks(world, sum(lat))
        out[name] = {"value": round(world * steps / (t / 1e3), 3), "unit": "solves/s",
                     "ms_per_step": round(t / steps, 3), "iters": it, "levels": nlev}
    return out


def time_config(args, world, flush, stream, A, b, x, opts, steps, warmup):
    """Setup + solve steps of one configuration: per-step CUDA events around the setup and
    around the solve (L2 flushed before every step, outside the events)."""
    import torch

    from paper_1209_5421_gb300 import amg

    def step(mid=None):
        h = amg.Hierarchy(*A, **opts)
        if mid is not None:
            mid.record(stream)
        _, it, rr, st = h.solve(b, args.tol, x=x)
        h.close()
        if st != amg.OK:
            raise RuntimeError(f"solve failed: status {st}, relres {rr}")
        return it, rr

    for _ in range(warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    barrier(world)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    its, rrs = [], []
    for k in range(steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        it, rr = step(ev[k][1])
        ev[k][2].record(stream)
        its.append(it)
        rrs.append(rr)
    torch.cuda.synchronize()
    barrier(world)
    lat = [e[0].elapsed_time(e[2]) for e in ev]
    total = max_over_ranks(world, sum(lat))
    return {"value": round(world * steps / (total / 1e3), 3), "unit": "solves/s",
            "ms_per_step": round(total / steps, 3),
            "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3),
                           "p99": round(float(np.percentile(lat, 99)), 3)},
            "setup_ms": round(statistics.median(e[0].elapsed_time(e[1]) for e in ev), 3),
            "solve_ms": round(statistics.median(e[1].elapsed_time(e[2]) for e in ev), 3),
            "iters": its[-1], "relres": float(max(rrs)), "steps": steps}


def golden_oracle_iters(name, tol):
    """The FP64 oracle's outer iterations for a workload, from the stored golden counts."""
    p = os.path.join(ROOT, "tests", "golden", "oracle_counts.txt")
    try:
        for line in open(p):
            f = line.split()
            if f and not line.startswith("#") and f[0] == name and float(f[1]) == tol:
                return int(f[2])
    except OSError:
        pass
    return None


def run_small_latency(args, world, flush, dev, stream):
    """The 65 x 65-node jittered P1 Poisson (3,969 unknowns, load vector of f = 1, auxiliary
    grid 64 x 64), the plain FP64 method (FP64 cycle, flexible-CG outer), one system per step:
    the latency case. Error against the FP64 oracle's solution of the same system."""
    import torch

    from oracle import oracle
    from paper_1209_5421_gb300 import amg
    from paper_1209_5421_gb300.meshes import workload

    prob, aux = workload("quasi_uniform_65")
    td = lambda a: torch.as_tensor(a).to(dev)  # noqa: E731
    A = [td(a) for a in (prob.rowptr, prob.col, prob.val, prob.x, prob.y)]
    b = td(prob.b)
    x = torch.empty_like(b)
    res = time_config(args, world, flush, stream, A, b, x,
                      dict(aux_level=aux, cycle_prec=amg.FP64, outer=amg.OUTER_FCG),
                      steps=max(20, args.steps), warmup=max(3, args.warmup))
    xg = x.cpu().numpy()
    oracle.build()
    O = oracle.Hierarchy.from_problem(prob, aux_level=aux)
    xo, ito, _, _ = O.solve(prob.b, args.tol)
    return {"workload": "quasi_uniform_65", "unknowns": prob.n, "nnz": prob.nnz,
            "aux_level": aux, "method": "FP64 AMLI-cycle, flexible-CG outer (plain method)",
            **res, "iters_oracle": ito, "err_vs_oracle": rel_err(xg, xo)}


def run_graded(args, world, flush, dev, stream):
    """The graded workload: 1449 x 1449-node P1 Poisson with x -> x^2, y -> y^2, jitter 0.1h
    and kappa log-uniform in [0.1, 10] on 16 x 16 blocks (2,093,809 unknowns, L = 10 by the
    depth rule): FP32 cycle with FP64 FGMRES, and the plain FP64 method beside it; the
    oracle's iteration count from the stored golden counts; per-op rates of the finest
    level's block Gauss-Seidel colours from a profiling pass."""
    import torch

    from paper_1209_5421_gb300 import amg
    from paper_1209_5421_gb300.meshes import workload

    prob, aux = workload("graded_1449")
    td = lambda a: torch.as_tensor(a).to(dev)  # noqa: E731
    A = [td(a) for a in (prob.rowptr, prob.col, prob.val, prob.x, prob.y)]
    b = td(prob.b)
    x = torch.empty_like(b)
    steps = max(2, min(args.steps, 4))
    out = {"workload": "graded_1449", "unknowns": prob.n, "nnz": prob.nnz,
           "iters_oracle": golden_oracle_iters("graded_1449", args.tol)}
    for name, o in (("fp32_fgmres", dict(aux_level=aux, cycle_prec=amg.FP32,
                                         outer=amg.OUTER_FGMRES)),
                    ("fp64_fcg", dict(aux_level=aux, cycle_prec=amg.FP64, outer=amg.OUTER_FCG))):
        out[name] = time_config(args, world, flush, stream, A, b, x, o, steps=steps,
                                warmup=max(1, min(args.warmup, 2)))
    if not args.no_profile:
        h = amg.Hierarchy(*A, aux_level=aux, cycle_prec=amg.FP32, outer=amg.OUTER_FGMRES)
        h.profile(2)
        flush.fill_(0.0)
        h.solve(b, args.tol, x=x)
        ks = h.profile_read()
        nl = h.nlev
        info = [h.level_info(l) for l in range(nl)]
        agg = h.level(0)["agg"]
        h.close()
        out["levels"] = nl
        # the finest level's block Gauss-Seidel: unknowns per aggregate (one thread a block)
        per = np.bincount(agg)
        out["fine_block_rows"] = {"max": int(per.max()), "mean": round(float(per.mean()), 2),
                                  "blocks": int(len(per))}
        out["kernels"] = sorted(
            [{"name": k["name"], "launches": k["launches"], "ms": round(k["ms"], 4),
              "GBps": round(k["bytes"] / (k["ms"] / 1e3) / 1e9, 1) if k["ms"] > 0 else None}
             for k in ks], key=lambda d: -d["ms"])[:10]
        out["level_rows"] = [int(i["n"]) for i in info]
    return out


def serve_matrices(count=24, seed=11):
    """The served stream's matrices: `count` P1 Poisson systems with unknowns log-uniform in
    [1e3, 4e6], alternately quasi-uniform (jitter 0.2h) and graded (x -> x^2, y -> y^2,
    jitter 0.1h, kappa on 16 x 16 blocks), each with its own mesh seed."""
    from paper_1209_5421_gb300.meshes import p1_poisson

    rng = np.random.default_rng(seed)
    unknowns = np.exp(rng.uniform(np.log(1e3), np.log(4e6), count))
    sides = np.rint(np.sqrt(unknowns)).astype(int) + 2
    mats = []
    for k, m in enumerate(sides):
        if k % 2:
            mats.append(p1_poisson(int(m), jitter=0.1, graded=True, kappa_blocks=16,
                                   seed=100 + k, rhs="normal"))
        else:
            mats.append(p1_poisson(int(m), jitter=0.2, seed=100 + k, rhs="normal"))
    return mats


def run_served_rate(args, local, mats, rate, nreq, seed):
    """One rate of the served form: a fresh server, a Poisson stream of `nreq` requests at
    `rate` req/s; 30% of the requests reuse a matrix already seen with a new N(0,1) rhs, the
    others bring the next new matrix (while any is left). Latency = completion - arrival."""
    from paper_1209_5421_gb300.serve import Server

    rng = np.random.default_rng(seed)
    S = Server(budget_bytes=150 << 30, device=local, large_unknowns=args.serve_large)
    for k, p in enumerate(mats):
        S.register(k, p.rowptr, p.col, p.val, p.x, p.y)
    seen, nxt, reqs = [], 0, []
    for i in range(nreq):
        if seen and (rng.random() < 0.3 or nxt == len(mats)):
            key = seen[rng.integers(len(seen))]
        else:
            key = nxt
            nxt += 1
            seen.append(key)
        reqs.append((key, rng.standard_normal(mats[key].n), float(rng.exponential(1.0 / rate))))
    t0 = time.perf_counter()
    handles = []
    for key, b, gap in reqs:
        handles.append(S.submit(key, b, args.tol))
        time.sleep(gap)
    offered_s = time.perf_counter() - t0
    S.drain()
    wall = time.perf_counter() - t0
    st = S.stats()
    S.close()
    bad = [r.status for r in handles if r.status != 0]
    if bad:
        raise RuntimeError(f"served at {rate} req/s: failed statuses {sorted(set(bad))}")
    return {"rate_offered": rate, "offered_req_per_s": round(nreq / offered_s, 2),
            "value": round(st["solves_per_s"], 2), "unit": "solves/s",
            "latency_ms": {"p50": round(st["p50_ms"], 2), "p99": round(st["p99_ms"], 2)},
            "requests": nreq, "wall_s": round(wall, 2), "setups": st["setups"],
            "group_setups": st.get("group_setups", 0),
            "evictions": st["evictions"], "batches": st["batches"],
            "large_lane_solves": st["large_lane"],
            "max_resident_bytes": st["max_resident_bytes"],
            "relres_max": max(r.relres for r in handles)}


def run_served(args, local):
    """The served form, swept over offered rates: the same matrices (quasi-uniform and graded,
    1e3..4e6 unknowns) and a fresh continuous-batching server per rate (HBM budget 150 GB)."""
    mats = serve_matrices()
    rates = [float(r) for r in args.serve_rates.split(",")]
    per_rate = [run_served_rate(args, local, mats, r, args.serve_requests, 11 + k)
                for k, r in enumerate(rates)]
    return {
        "workload": f"{args.serve_requests} requests per rate, Poisson arrivals; "
                    f"{len(mats)} matrices of 1e3..4e6 unknowns (log-uniform), quasi-uniform "
                    "and graded alternately, 30% reuse",
        "method": "FP32 AMLI-cycle; batch lane FP64 flexible CG (one CTA per system), "
                  f"large lane (> {args.serve_large} unknowns) FP64 FGMRES on the whole GPU",
        "unknowns": [int(m.n) for m in mats],
        "large_lane_unknowns": args.serve_large,
        "budget_bytes": 150 << 30,
        "rates": per_rate,
    }


def run_ours(args, world, rank, local):
    import torch

    from paper_1209_5421_gb300 import amg
    from paper_1209_5421_gb300.meshes import workload

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prob, aux = workload(args.workload)
    prec = amg.FP32 if args.prec == "fp32" else amg.FP64
    outer = amg.OUTER_FGMRES if args.outer == "fgmres" else amg.OUTER_FCG
    opts = dict(aux_level=aux, cycle_prec=prec, outer=outer)
    td = lambda a: torch.as_tensor(a).to(dev)  # noqa: E731
    A = [td(a) for a in (prob.rowptr, prob.col, prob.val, prob.x, prob.y)]
    b = td(prob.b)
    x = torch.empty_like(b)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    launch_total = [0]

    def step(o=opts, mid=None):
        h = amg.Hierarchy(*A, **o)
        if mid is not None:  # setup returns once its work is done: the setup / solve split
            mid.record(stream)
        _, it, rr, st = h.solve(b, args.tol, x=x)
        su, so = h.launch_counts()
        launch_total[0] += su + so
        h.close()
        if st != amg.OK:
            raise RuntimeError(f"solve failed: status {st}, relres {rr}")
        return it, rr

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    launch_total[0] = 0
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    mids = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    iters = []
    barrier(world)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            it, rr = step(mid=mids[k])
            ends[k].record(stream)
            iters.append(it)
        torch.cuda.synchronize()
    barrier(world)
    lat = [s.elapsed_time(e) for s, e in zip(starts, ends)]  # ms
    setup_ms = statistics.median(s.elapsed_time(m) for s, m in zip(starts, mids))
    solve_ms = statistics.median(m.elapsed_time(e) for m, e in zip(mids, ends))
    x_head = x.cpu().numpy().copy()
    total_ms = max_over_ranks(world, sum(lat))
    value = world * args.steps / (total_ms / 1e3)
    launches_timed = launch_total[0]

    # ---- the plain FP64 method (FP64 cycle, flexible-CG outer) on the same workload
    fp64_line = None
    if not args.no_fp64_line and not (prec == amg.FP64 and outer == amg.OUTER_FCG):
        o64 = dict(aux_level=aux, cycle_prec=amg.FP64, outer=amg.OUTER_FCG)
        for _ in range(max(1, args.warmup)):
            flush.fill_(1.0)
            step(o64)
        torch.cuda.synchronize()
        lat64, its64 = [], []
        for k in range(args.steps):
            flush.fill_(float(k))
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            it64, _ = step(o64)
            ev1.record(stream)
            its64.append(it64)
            torch.cuda.synchronize()
            lat64.append(ev0.elapsed_time(ev1))
        t64 = max_over_ranks(world, sum(lat64))
        fp64_line = {"value": round(world * args.steps / (t64 / 1e3), 3), "unit": "solves/s",
                     "ms_per_step": round(t64 / args.steps, 3), "iters": its64[-1],
                     "method": "FP64 AMLI-cycle, flexible-CG outer"}
        x64 = x.cpu().numpy().copy()

    # ---- e2e: the C ABI with pinned host buffers (H2D of inputs, D2H of x inside the step)
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.as_tensor(a).pin_memory()  # noqa: E731
        Ah = [pin(a) for a in (prob.rowptr, prob.col, prob.val, prob.x, prob.y)]
        bh = pin(prob.b)
        xh = torch.empty_like(bh).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in Ah) + bh.numel() * bh.element_size()
        d2h = xh.numel() * xh.element_size()

        def step_host():
            h = amg.Hierarchy(*Ah, **opts)
            _, it, rr, st = h.solve(bh, args.tol, x=xh)
            h.close()
            if st != amg.OK:
                raise RuntimeError(f"solve failed: status {st}")

        for _ in range(max(1, args.warmup)):
            step_host()
        torch.cuda.synchronize()
        barrier(world)
        el = 0.0
        for k in range(args.steps):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            step_host()
            el += time.perf_counter() - t0
        barrier(world)
        el = max_over_ranks(world, el)
        e2e = {"value": world * args.steps / el, "unit": "solves/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    # ---- profiling pass: per-kernel CUDA-event durations and algorithmic bytes
    roofline = None
    kernels = None
    if not args.no_profile:
        h = amg.Hierarchy(*A, **opts)
        h.profile(2)  # per kernel and per grid op; the shared-memory tail timed as a whole
        flush.fill_(0.0)
        torch.cuda.synchronize()
        h.solve(b, args.tol, x=x)
        kernels = h.profile_read()
        h.close()
        peak, peak_kind = measured_peak_hbm()
        whole = [k for k in kernels if not k["name"].startswith(("in_cycle:", "in_tail:"))]
        dom = max(whole, key=lambda k: k["ms"])
        ach = dom["bytes"] / dom["launches"] / (dom["ms"] / dom["launches"] / 1e3) / 1e9
        roofline = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(ach / peak, 4),
                    "traffic": recorded_traffic(args.workload, args.prec),
                    "kernel": dom["name"], "peak_source": f"{peak_kind} (MEASURED_PEAKS hbm_gbs)",
                    "bytes_per_launch": dom["bytes"] / dom["launches"],
                    "ms_per_launch": dom["ms"] / dom["launches"],
                    "launches_in_solve": dom["launches"]}

    small = None if args.no_small else run_small_latency(args, world, flush, dev, stream)
    graded = None if args.no_graded else run_graded(args, world, flush, dev, stream)
    batched = None if args.no_batch else run_batched(args, world, flush, dev, stream)
    served = None if (args.no_serve or rank != 0) else run_served(args, local)
    octree = None if args.no_octree else run_octree(args, world, flush, dev, stream)

    out = None
    if rank == 0:
        cpu = None
        err_vs_oracle = None
        if not args.no_cpu and world == 1:
            c = cpu_oracle_baseline(prob, aux, args.tol)
            tot = c["setup_s"] + c["solve_s"]
            cpu = {"value": 1.0 / tot, "unit": "solves/s", "cores": 1, "kind": "oracle",
                   "sample": f"one full oracle setup+solve of {args.workload} "
                             f"({c['iters']} iterations, {tot:.1f} s)"}
            err_vs_oracle = rel_err(x_head, c["x"])
            if fp64_line is not None:
                fp64_line["err_vs_oracle"] = rel_err(x64, c["x"])
                fp64_line["iters_oracle"] = c["iters"]
        lat_sorted = sorted(lat)
        out = {
            "metric": METRIC, "value": round(value, 3), "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == amg.FP64 else "f32-cycle/f64-outer",
            "method": ("FP32" if prec == amg.FP32 else "FP64") + " AMLI-cycle, "
                      + ("restarted flexible GMRES(30)" if outer == amg.OUTER_FGMRES else "flexible CG")
                      + " outer in FP64",
            "data": "synthetic",
            "config": {"workload": args.workload, "unknowns": prob.n, "nnz": prob.nnz,
                       "aux_level": aux, "tol": args.tol, "iters": iters[-1],
                       "l2": "flushed (256 MiB write) before every timed step",
                       "parallelism": f"replicas{world}"},
            "setup_ms": round(setup_ms, 3), "solve_ms": round(solve_ms, 3),
            "iters": iters[-1],
            "err_vs_oracle": err_vs_oracle,
            "latency_ms": {"p50": round(float(np.percentile(lat_sorted, 50)), 3),
                           "p99": round(float(np.percentile(lat_sorted, 99)), 3)},
            "clocks": clk.summary(),
            "e2e": e2e,
            "gpu_launches": launches_timed,
            "fp64_plain": fp64_line,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "small_fp64": small,
            "graded": graded,
            "batched": batched,
            "served": served,
            "octree": octree,
        }
        if kernels:
            out["kernels"] = sorted(
                [{"name": k["name"], "launches": k["launches"], "ms": round(k["ms"], 4),
                  "GBps": round(k["bytes"] / (k["ms"] / 1e3) / 1e9, 1) if k["ms"] > 0 else None}
                 for k in kernels], key=lambda d: -d["ms"])[:16]
        print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    world, rank, local = dist_setup()
    try:
        if args.impl == "reference":
            return run_reference(args, world, rank)
        return run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
