"""The product path has no CPU fallback and never touches the oracle.

Runs without a GPU. Setup and solve exist only as CUDA kernels behind the C ABI: on a machine
without a usable GPU a valid setup must fail with a CUDA status (nothing is computed on the
host), a missing library must raise at load time, and importing the package's modules must
not load the CPU oracle.
"""
import os
import subprocess
import sys

import pytest

from paper_1209_5421_gb300 import amg, build, meshes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_valid_setup_without_a_gpu_fails_with_a_cuda_status(libpath):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the setup would run on it")
    p = meshes.p1_poisson(17, jitter=0.2, seed=0)
    with pytest.raises(amg.AmgError) as e:
        amg.Hierarchy.from_problem(p)
    assert e.value.status == amg.ERR_CUDA


def test_missing_library_raises(monkeypatch):
    monkeypatch.setattr(amg, "_lib", None)
    monkeypatch.setattr(amg, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "libamg_gb300.so"))
    with pytest.raises(RuntimeError, match="missing"):
        amg.lib()


def test_product_modules_do_not_load_the_oracle():
    code = ("import sys\n"
            "import paper_1209_5421_gb300.amg, paper_1209_5421_gb300.meshes\n"
            "import paper_1209_5421_gb300.serve, paper_1209_5421_gb300.cli\n"
            "import paper_1209_5421_gb300.build\n"
            "bad = [m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')]\n"
            "assert not bad, bad\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
