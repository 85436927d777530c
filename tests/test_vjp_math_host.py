"""The adjoint's point-wise reverse passes (HLLC + Einfeldt, WENO5-JS),
compiled for the host with nvcc, against central differences of the forward
functions.  CPU only (needs nvcc, not a GPU)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reverse_passes_match_central_differences(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "vjp_math_check"
    src = os.path.join(ROOT, "tests", "host_checks", "vjp_math_check.cu")
    inc = os.path.join(ROOT, "paper_2203_13760_gb300", "csrc")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O2", "-x", "cu", "-I", inc,
                    src, "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    errs = {line.split()[0]: float(line.split()[-1]) for line in out.strip().splitlines()}
    assert errs["hllc"] < 1e-6, out
    assert errs["weno"] < 1e-6, out
