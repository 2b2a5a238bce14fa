"""Integer-pipe float/double conversions of the CUDA path, checked on the host.

The kernels convert between float and double with integer operations (the
FP64 pipe of GB300 is slow and would also run the hardware conversions).  The
same functions compile as host code, so nvcc builds a small host program that
compares them bit for bit with the C casts: IEEE round-to-nearest-even for
double -> float in the float normal range, exact float -> double.
"""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_conversions_match_c_casts(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "conversions"
    subprocess.run([nvcc, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2301_07457_gb300", "csrc"),
                    "-o", str(exe), os.path.join(ROOT, "tests", "native", "conversions.cu")],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok ")
