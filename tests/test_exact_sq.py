"""The fused kernel's integer exact-square routine (csrc/exact_sq.h), compiled
for the host with g++ and compared bit for bit with (double)x * (double)x."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_exact_square_bits(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    exe = tmp_path / "exact_sq_check"
    src = os.path.join(ROOT, "tests", "cpp", "exact_sq_check.cpp")
    inc = os.path.join(ROOT, "paper_2305_14398_gb300", "csrc")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", inc, src, "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0" in r.stdout
