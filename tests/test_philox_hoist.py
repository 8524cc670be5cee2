"""The hoisted Philox forms of the kernels (PhiloxS, PhiloxT in csrc/stf_device.cuh), compiled as
host code with nvcc and run on the CPU: they return exactly philox() of the same counter on
400,000 random counters and keys, and philox() gives the Random123 known answer for the zero
counter and key."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_hoisted_philox_equals_philox(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "philox_hoist_check")
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"),
                    "-o", exe, os.path.join(HERE, "host", "philox_hoist_check.cu")], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0 kat 1" in r.stdout
