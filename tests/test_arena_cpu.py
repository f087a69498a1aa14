"""Host-only check of the batching engine's arena allocator (csrc/fwi_arena.h): compiles
tests/native/arena_check.cpp with g++ and runs it (random allocations and releases against
an independent byte map; first fit, alignment, disjointness, coalescing)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1804_01184_gb300", "csrc")


def test_arena_first_fit_and_coalescing(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "arena_check")
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, os.path.join(HERE, "native", "arena_check.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "arena ok" in r.stdout, r.stdout + r.stderr
