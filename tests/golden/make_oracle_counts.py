"""Writes oracle_counts.txt: the FP64 oracle's outer iteration counts and true relative
residuals on workloads whose oracle solve is too slow to repeat inside a test.

Calls only oracle/ (and the seeded input generators): no value here comes from the CUDA
path. Run from the repository root: python tests/golden/make_oracle_counts.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402
from paper_1209_5421_gb300.meshes import workload  # noqa: E402

# (workload, tolerance): the oracle's plain method (FP64 cycle, flexible CG outer, Alg. 1)
CASES = [("quasi_uniform_65", 1e-8), ("graded_1449", 1e-8)]


def main():
    oracle.build()
    lines = ["# Outer iterations (B^ applications) and true relative residual of the FP64 oracle,",
             "# written by tests/golden/make_oracle_counts.py (oracle/ only).",
             "# workload tol iterations relres"]
    for name, tol in CASES:
        prob, aux = workload(name)
        h = oracle.Hierarchy.from_problem(prob, aux_level=aux)
        x, it, rr, st = h.solve(prob.b, tol)
        assert st == oracle.OK, (name, st)
        true = np.linalg.norm(prob.b - prob.to_scipy() @ x) / np.linalg.norm(prob.b)
        lines.append(f"{name} {tol:g} {it} {true:.6e}")
        print(lines[-1], flush=True)
    with open(os.path.join(HERE, "oracle_counts.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
