"""The 3D direct kernel's row partition, compiled from d3.cuh for the host and run here (no GPU): interior and
edge rows cover every row of the grid once (tests/host_rows3.cu)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_interior_and_edge_rows_partition_the_grid():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "host_rows3")
        cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "--expt-relaxed-constexpr",
               "-I" + os.path.join(ROOT, "include"), "-I" + os.path.join(ROOT, "paper_1704_04413_gb300", "csrc"),
               os.path.join(ROOT, "tests", "host_rows3.cu"), "-o", exe]
        subprocess.run(cmd, check=True, capture_output=True)
        out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout
    assert "partition ok" in out.stdout
