"""Host check of the ray-segment seek used by the traversal kernels (compiled with nvcc as host
code; no GPU needed): the closed-form state at every segment start equals plain stepping."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_segment_seek_matches_stepping():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "dda_seek_check")
        src = os.path.join(ROOT, "tests", "dda_seek_check.cu")
        inc = os.path.join(ROOT, "paper_1611_03631_gb300", "csrc")
        subprocess.run([nvcc, "-O2", "-std=c++17", "-I", inc, src, "-o", exe], check=True, capture_output=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stdout + r.stderr
        assert r.stdout.startswith("ok")
