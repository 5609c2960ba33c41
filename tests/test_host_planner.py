"""Host-side planner checks (no GPU): compiles tests/host/planner_check.cu
against the library's planning header and runs it.  It replays the striped
kernel's lane schedule for random bands and every variant and verifies the
period, ring size and step count the planner computes in closed form, the
launch-class ordering, the kernel's O(1) row step of the band DDA, the exact
in-band cell count the kernel reports (floor sums) against row-by-row sums,
and the host worker pool's parallel loops."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="needs nvcc (host code only)")
def test_schedule_and_classes():
    src = os.path.join(ROOT, "tests", "host", "planner_check.cu")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "planner_check")
        subprocess.check_call(["nvcc", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I",
                               os.path.join(ROOT, "paper_2310_05037_gb300", "csrc"), src, "-o", exe])
        out = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    print(out.stdout)
    assert out.returncode == 0, out.stdout[-3000:]
    assert "fails 0" in out.stdout
