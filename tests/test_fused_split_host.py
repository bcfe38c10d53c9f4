"""Host logic of the fused sketch pass, without a GPU: its tile split over
the CTAs and its partial-slot layout (the helpers of csrc/fused.cu compiled
for the host by nvcc; no kernel runs).  Every tile has one owner whose
range holds it, the ranges tile the grid, the slot indices the CTAs write
never collide and stay inside the workspace, and the sum kernel lists only
written slots -- over tall, wide, ragged and one-tile shapes, one- and
two-sided passes, and 1 to 152 CTAs."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_fused_split_and_slots(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "fused_split_check")
    src = os.path.join(ROOT, "tests", "host", "fused_split_check.cu")
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17",
           "--expt-relaxed-constexpr", "-O1", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(ROOT, "paper_1505_04650_gb300", "csrc"), src,
           "-o", exe, "-lcuda"]
    b = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert b.returncode == 0, b.stderr[-3000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
