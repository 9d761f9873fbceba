"""Exhaustive host-side check of the kernels' sector indexers and gate orbit
enumerations (CPU only: the same header code compiled for the host).

Every sector tuple's rank and unrank, every number-conserving move's rank
change, and the exact-once coverage of the sector by each gate's orbits are
compared with brute-force lexicographic enumeration."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_index_arithmetic_exhaustive():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc) and shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "index_check")
        src = os.path.join(ROOT, "tests", "index_check.cu")
        inc = ["-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2606_05297_gb300", "csrc")]
        subprocess.run([nvcc, "-std=c++17", "-O1", *inc, src, "-o", exe], check=True, capture_output=True, text=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stdout + r.stderr
        assert "OK" in r.stdout
