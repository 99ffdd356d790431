"""The shared-memory and TMEM plans of the two tcgen05 kernels (the bottleneck kernel and the
H-transform kernel) over a sweep of about 12 M shape/form combinations: every accepted plan keeps
its regions in bounds, ordered and aligned, its MMA shapes legal and its TMEM columns within the
allocation (tests/tcgen05_plan_check.cu, compiled with nvcc and run on the host; no GPU)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_tcgen05_plans_are_in_bounds_aligned_and_legal(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "tcgen05_plan_check"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O1", "-std=c++17",
                    "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_1510_03298_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "tcgen05_plan_check.cu"), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "failures 0" in r.stdout, r.stdout
