"""Host-side logic of bench.py (no GPU): the ncu traffic bookkeeping.

The roofline's `traffic` comes from profiles/step_kernel_traffic.json only
while the sources its kernel is compiled from are those the capture was
taken with; any edit of one of them makes it null.
"""
import json
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_every_profiled_kernel_names_existing_sources():
    csrc = os.path.join(ROOT, "paper_1804_02418_gb300", "csrc")
    for key, files in bench.KERNEL_SOURCES.items():
        for f in files:
            assert os.path.exists(os.path.join(csrc, f)), (key, f)


def _fake_root(tmp_path):
    root = tmp_path / "r"
    shutil.copytree(os.path.join(ROOT, "paper_1804_02418_gb300", "csrc"),
                    root / "paper_1804_02418_gb300" / "csrc")
    (root / "profiles").mkdir()
    return root


def test_traffic_is_used_only_while_the_sources_match(tmp_path, monkeypatch):
    root = _fake_root(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    entry = {"dram_bytes_per_launch": 123456, "source_hash": bench.source_hash("f32")}
    with open(root / "profiles" / "step_kernel_traffic.json", "w") as f:
        json.dump({"f32": entry, "massive_f32": dict(entry, source_hash=bench.source_hash("massive_f32"))}, f)
    assert bench.ncu_traffic("f32") == 123456
    assert bench.ncu_traffic("massive_f32") == 123456
    assert bench.ncu_traffic("f16dev") is None            # no capture for it
    assert bench.ncu_traffic("no_such_kernel") is None
    # a change to a source of the massive kernel leaves the massless entry valid
    with open(root / "paper_1804_02418_gb300" / "csrc" / "massive.cu", "a") as f:
        f.write("\n// edited\n")
    assert bench.ncu_traffic("massive_f32") is None
    assert bench.ncu_traffic("f32") == 123456
    with open(root / "paper_1804_02418_gb300" / "csrc" / "kernels.cuh", "a") as f:
        f.write("\n// edited\n")
    assert bench.ncu_traffic("f32") is None


def test_host_copies_is_at_least_one():
    assert bench.host_copies() >= 1
