"""Host-only checks of the serving loop's bookkeeping: the device-memory
arena and the scheduler's admission (arrival order, memory budget, slots),
step packing (quota, task groups, root-find units) and release rules.  The
C++ header is compiled with g++ here; no GPU is involved."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1105_4747_gb300", "csrc")
SRC = os.path.join(ROOT, "tests", "serve_sched_check.cpp")

CHECKS = ["arena_random", "budget_and_fifo", "slots", "quota_interleave", "units_cover", "random_loop"]


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("sched") / "serve_sched_check")
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-I", CSRC, SRC, "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    return r


@pytest.mark.parametrize("name", CHECKS)
def test_sched(run, name):
    assert f"PASS {name}" in run.stdout, run.stdout + run.stderr
