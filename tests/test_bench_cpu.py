"""bench.py's measured-traffic bookkeeping (no GPU): the committed ncu DRAM figures are used
only while the kernel sources they were taken from are unchanged, and are scaled to the
launch's shots."""
import importlib.util
import json
import os
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench(root):
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(root, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    b.ROOT = root
    return b


@pytest.fixture
def tree(tmp_path):
    """A copy of the files the bookkeeping reads: bench.py, the step-kernel sources, traffic.json."""
    for rel in ("bench.py", "profiles/traffic.json"):
        os.makedirs(tmp_path / os.path.dirname(rel), exist_ok=True)
        shutil.copy(os.path.join(ROOT, rel), tmp_path / rel)
    csrc = tmp_path / "paper_1804_01184_gb300" / "csrc"
    os.makedirs(csrc)
    for f in ("fwi_warp.cuh", "fwi_stream.cuh", "fwi_kernels.cuh"):
        shutil.copy(os.path.join(ROOT, "paper_1804_01184_gb300", "csrc", f), csrc / f)
    return tmp_path


def test_traffic_scales_with_shots_and_lapses_when_a_kernel_changes(tree):
    b = load_bench(str(tree))
    t = json.load(open(tree / "profiles" / "traffic.json"))
    k = t["kernels"]["k_fwd_warp"]
    assert b.measured_traffic("k_fwd_warp", k["shots_per_launch"]) == k["dram_bytes_per_launch"]
    assert b.measured_traffic("k_fwd_warp", k["shots_per_launch"] / 2) == int(k["dram_bytes_per_launch"] / 2)
    assert b.measured_traffic("k_no_such_kernel", 64) is None
    with open(tree / "paper_1804_01184_gb300" / "csrc" / "fwi_warp.cuh", "a") as f:
        f.write("\n// changed\n")
    assert b.measured_traffic("k_fwd_warp", 64) is None


def test_fborn_traffic_file_names_the_kernels_the_bench_looks_up():
    t = json.load(open(os.path.join(ROOT, "profiles", "traffic_fborn.json")))
    assert len(t["kernel_source_sha256"]) == 64
    assert set(t["kernels"]) == {"k_fb_model_tc", "k_fb_grad"}
    assert all(k["dram_bytes_per_launch"] > 1.5e9 for k in t["kernels"].values())   # the 1.55 GB of tables
