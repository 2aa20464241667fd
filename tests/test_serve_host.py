"""Host logic of the request server (no GPU): the device arena's allocator
and the step planner, compiled from the library's own header into a small
C++ test program (tests/host/serve_sched_test.cpp)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_arena_and_step_planner(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "serve_sched_test")
    subprocess.run([gxx, "-std=c++17", "-O1", "-Wall", "-Werror",
                    "-I", os.path.join(ROOT, "paper_2403_06777_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host", "serve_sched_test.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "ok"
