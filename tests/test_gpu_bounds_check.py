"""GPU: the bounds-checking build of the library (index checks that set a flag, never trap).

The variant libamg_gb300_bc.so is built with -DAMG_BOUNDS_CHECK: every gather of the cycle's
and the batch kernel's ops checks its index against the vector's length, skips an access
outside it and sets a flag that amg_debug_bounds_flags reads. A parity case runs on it in a
child process (the binding loads the variant through AMG_GB300_LIBRARY): the same results as
the oracle, and no flag set. The normal build reports that it has no checks.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np
from oracle import oracle
from paper_1209_5421_gb300 import amg
from paper_1209_5421_gb300.meshes import p1_poisson
assert amg.LIB_PATH.endswith("libamg_gb300_bc.so"), amg.LIB_PATH
assert amg.bounds_flags() == 0
cases = [dict(n=33, jitter=0.2, seed=1, rhs="normal"),
         dict(n=65, jitter=0.1, graded=True, kappa_blocks=16, seed=2, rhs="normal"),
         dict(n=97, jitter=0.2, seed=6, rhs="normal")]
for spec in cases:
    p = p1_poisson(**spec)
    for kw in ({}, dict(cycle_prec=amg.FP32, outer=amg.OUTER_FGMRES)):
        G = amg.Hierarchy.from_problem(p, **kw)
        x, it, rr, st = G.solve(p.b, 1e-8)
        O = oracle.Hierarchy.from_problem(p)
        xo, ito, _, _ = O.solve(p.b, 1e-8)
        assert st == amg.OK, (spec, kw, st)
        if not kw:  # the plain FP64 method: the oracle's iteration count within one
            assert abs(it - ito) <= 1, (spec, it, ito)
        A = p.to_scipy()
        assert np.linalg.norm(p.b - A @ x) <= 1e-8 * np.linalg.norm(p.b)
        assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)
        G.close()
B = amg.Batch.from_problems([p1_poisson(**c) for c in cases], cycle_prec=amg.FP32)
rhs = np.concatenate([p1_poisson(**c).b for c in cases])
x, it, rr, st = B.solve(rhs, 1e-8)
assert (st == amg.OK).all()
B.close()
flags = amg.bounds_flags()
assert flags == 0, flags
print("bounds-checked parity ok")
"""


def test_bounds_checked_build_parity():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    from paper_1209_5421_gb300 import amg, build

    path = build.build(bounds_check=True)
    env = dict(os.environ, AMG_GB300_LIBRARY=path)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    assert "bounds-checked parity ok" in r.stdout
    # the normal build has no checks and says so
    build.build()
    with pytest.raises(amg.AmgError) as ei:
        amg.bounds_flags()
    assert ei.value.status == amg.ERR_UNSUPPORTED
