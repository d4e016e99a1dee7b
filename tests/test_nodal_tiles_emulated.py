"""Host emulation of the tiled nodal multigrid kernels.

``tests/native/nodal_tiles_emu.cpp`` compiles ``csrc/nodal_tiles.cuh`` with the host
compiler (the CUDA qualifiers expand to nothing there) and runs the kernels CTA by CTA,
one host thread per CUDA thread, the threads of a CTA taking turns between barriers in a
fixed order, under AddressSanitizer with the shared memory beyond each launch's size
poisoned and the rest filled with NaN.  It checks that the register-blocked FP32 steps
(``k_node_down_rb`` / ``k_node_up_rb``, every launch shape the autotuner offers) give the
results of ``k_node_down`` / ``k_node_up`` bit for bit, in ascending and descending
thread order (a read of a word another thread writes in the same barrier interval would
make the two orders differ), on ragged levels, at Gamma, at the zone corner and with two
Bloch vectors per launch.  It also runs the plain tiled steps with one, two and three
sweeps per side, in FP32 and FP64, against the same steps written over the whole level in
colour order: tiles whose halo lies inside the level agree bit for bit, the others to
rounding (their halos carry phase products of staged values).  The GPU tests compare the
kernels with one sweep per side against the oracle; two and three sweeps are checked here
only.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2304_00337_gb300", "csrc")
SRC = os.path.join(ROOT, "tests", "native", "nodal_tiles_emu.cpp")


def _cuda_include():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
    return inc if os.path.exists(os.path.join(inc, "cuda_runtime.h")) else None


def test_register_blocked_steps_match_the_tiled_steps(tmp_path):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("g++ or the CUDA headers not found")
    exe = str(tmp_path / "nodal_tiles_emu")
    cmd = [cxx, "-std=c++20", "-O1", "-g", "-fsanitize=address", "-fno-omit-frame-pointer", "-ffp-contract=off",
           "-fno-strict-aliasing", "-Wno-unknown-pragmas", "-pthread", "-I", CSRC, "-I", inc, SRC, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout[-3000:] + r.stderr[-3000:]
