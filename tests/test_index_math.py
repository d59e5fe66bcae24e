"""Index arithmetic of the kernels checked on the host: FastDiv (the
column of a flat element index for broadcast leaves) against integer
division, and the 128-byte shared-memory swizzle of the TMA tiles (a
permutation of each box; column reads conflict-free). tests/index_math.cu
includes the library's own headers and is compiled with nvcc for the CPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_index_math_on_host(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc"
                                    if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "index_math")
    csrc = os.path.join(ROOT, "paper_2604_22242_gb300", "csrc")
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O2", "-I", csrc,
           "-I", os.path.join(ROOT, "include"), os.path.join(HERE, "index_math.cu"), "-o", exe]
    p = subprocess.run(cmd, capture_output=True, text=True)
    assert p.returncode == 0, p.stderr[-3000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-3000:]
    assert "0 failures" in r.stdout
