"""Host-compiled check of the blocked site order of the packed FP32/FP16
storage (index permutation, inverse, hops with periodic wrap): runs on the CPU
through nvcc's host compiler, no GPU needed."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_blocked_site_order(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "blocked_geometry"
    subprocess.run([nvcc, "-std=c++17", "-O1", os.path.join(HERE, "host", "blocked_geometry.cu"), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout
