"""Host check of the integer-only binary32 <-> binary64 conversions of the CUDA path.

``csrc/fpconv.cuh`` compiles for host and device; ``tests/native/fpconv_check.cu``
compares it on the host with the compiler's IEEE conversions: every binary32 value
(binary32 -> binary64), and for binary64 -> binary32 random values at every exponent
around the binary32 range, the exact halfway patterns (ties to even) in the normal and
subnormal ranges, random bit patterns and the special values.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2304_00337_gb300", "csrc")
SRC = os.path.join(ROOT, "tests", "native", "fpconv_check.cu")


def test_conversions_match_ieee(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "fpconv_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, SRC, "-o", exe], check=True, capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
