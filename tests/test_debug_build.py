"""The bounds-checking debug build (-DJF_DEBUG_BOUNDS: every shared-memory,
ring and global index checked in the kernels, a device trace of the batch
work items) still compiles for the stage kernels and the batch driver.
CPU only: nvcc cross-compiles the translation units."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2203_13760_gb300 import _build  # noqa: E402

CSRC = os.path.join(ROOT, "paper_2203_13760_gb300", "csrc")


def _nvcc():
    try:
        return _build.nvcc()
    except RuntimeError:
        return None


def test_debug_bounds_build_compiles(tmp_path):
    cc = _nvcc()
    if cc is None:
        pytest.skip("nvcc not available")
    procs = []
    for unit in ("stage_f32.cu", "stage_f64.cu", "batch.cu"):  # compiled side by side
        cmd = [cc, *_build.ARCH, *_build.NVCC_FLAGS, *_build.PER_FILE_FLAGS.get(unit, []), "-DJF_DEBUG_BOUNDS",
               "-I", _build.INCLUDE, "-c", os.path.join(CSRC, unit), "-o", str(tmp_path / (unit + ".o"))]
        procs.append((unit, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for unit, p in procs:
        out, _ = p.communicate(timeout=900)
        assert p.returncode == 0, unit + ": " + out.decode(errors="replace")[-3000:]
