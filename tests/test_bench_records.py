"""The benchmark's use of the committed ncu record of a full-size pair-kernel launch (CPU only).

roofline.traffic and roofline.issue come from profiles/pair_kernel_traffic.json only while the record was
taken on the same kernel instance (path, proposal, tile shape) and on the sources as they are now; any other
instance, or an edited source, gives None rather than a stale number. The issue fraction is the record's
warp instructions over the launch time, against SMs x 4 schedulers x 1 warp instruction per clock.
"""
import json
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _record():
    return json.load(open(os.path.join(ROOT, "profiles", "pair_kernel_traffic.json")))


def test_record_matches_only_its_instance():
    d = _record()
    m = d["mixed"]
    shape = tuple(m["shape"])
    assert bench.kernel_traffic_record("mixed", m["proposal"], shape) == m["dram_bytes_per_launch"]
    assert bench.kernel_traffic_record("mixed", "bisect", shape) is None
    assert bench.kernel_traffic_record("mixed", m["proposal"], (64, 8)) is None
    assert bench.kernel_traffic_record("mixed", m["proposal"], shape + (16,)) is None  # the window instance
    f = d["fp64"]
    assert bench.kernel_traffic_record("fp64", f["proposal"], tuple(f["shape"])) == f["dram_bytes_per_launch"]


def test_record_is_dropped_when_a_source_changes(tmp_path, monkeypatch):
    # a copy of the tree's record and sources, one source edited: the record no longer applies
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    shutil.copy(os.path.join(ROOT, "profiles", "pair_kernel_traffic.json"), root / "profiles")
    csrc = root / "paper_2605_05543_gb300" / "csrc"
    shutil.copytree(os.path.join(ROOT, "paper_2605_05543_gb300", "csrc"), csrc,
                    ignore=shutil.ignore_patterns("*.o", "*.so"))
    monkeypatch.setattr(bench, "ROOT", str(root))
    m = _record()["mixed"]
    shape = tuple(m["shape"])
    assert bench.kernel_traffic_record("mixed", m["proposal"], shape) == m["dram_bytes_per_launch"]
    with open(csrc / m["sources"][0], "a") as fh:
        fh.write("\n")
    assert bench.kernel_traffic_record("mixed", m["proposal"], shape) is None
    assert bench.issue_roofline("mixed", m["proposal"], shape, 35.0, {"sm_mhz": 2070.0}, 152) is None


def test_issue_roofline_arithmetic():
    m = _record()["mixed"]
    shape = tuple(m["shape"])
    r = bench.issue_roofline("mixed", m["proposal"], shape, 40.0, {"sm_mhz": 2000.0}, 150)
    assert r["warp_instructions_per_launch"] == m["warp_instructions_per_launch"]
    assert r["achieved"] == pytest.approx(m["warp_instructions_per_launch"] / 0.040)
    assert r["peak"] == pytest.approx(150 * 4 * 2000e6)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # no clock record: the maximum SM clock
    assert bench.issue_roofline("mixed", m["proposal"], shape, 40.0, None, 150)["peak"] == pytest.approx(150 * 4 * 2070e6)
    # the FP64 record carries no instruction count
    f = _record()["fp64"]
    assert bench.issue_roofline("fp64", f["proposal"], tuple(f["shape"]), 600.0, {"sm_mhz": 2070.0}, 152) is None


def test_shape_key():
    assert bench.shape_key(None) is None
    t = dict(targets_per_block=128, sources_per_sum=32, history_window=0)
    assert bench.shape_key(t) == (128, 32)
    t["history_window"] = 16
    assert bench.shape_key(t) == (128, 32, 16)
