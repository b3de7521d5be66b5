"""The benchmark's use of a one-pass ncu record of a full-size pair-kernel launch (CPU only).

roofline.traffic and roofline.issue come from profiles/pair_kernel_traffic.json only while the record was
taken on the same kernel instance (path, proposal, tile shape) and on the sources as they are now; any other
instance, or an edited source, gives None rather than a stale number. The issue fraction is the record's
warp instructions over the launch time, against SMs x 4 schedulers x 1 warp instruction per clock. The
tests write their own record over a copy of the sources, so they hold whether or not the committed record
is current.
"""
import hashlib
import json
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

SOURCES = ["pair_mixed.cu", "emppp_api.cu", "emppp_internal.cuh"]


@pytest.fixture
def tree(tmp_path, monkeypatch):
    """A copy of the kernel sources with a record taken on them; bench.ROOT points at the copy."""
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    csrc = root / "paper_2605_05543_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in SOURCES + ["pair_fp64.cu"]:
        shutil.copy(os.path.join(ROOT, "paper_2605_05543_gb300", "csrc", name), csrc / name)

    def sha(names):
        h = hashlib.sha256()
        for n in names:
            h.update((csrc / n).read_bytes())
        return h.hexdigest()[:16]

    rec = {
        "mixed": {"proposal": "closed_form", "shape": [128, 32], "dram_bytes_per_launch": 1.4e9,
                  "warp_instructions_per_launch": 3.3e10, "sources": SOURCES, "sources_sha256_16": sha(SOURCES)},
        "fp64": {"proposal": "closed_form", "shape": [64, 8], "dram_bytes_per_launch": 2.3e9,
                 "sources": ["pair_fp64.cu", "emppp_api.cu", "emppp_internal.cuh"],
                 "sources_sha256_16": sha(["pair_fp64.cu", "emppp_api.cu", "emppp_internal.cuh"])},
    }
    (root / "profiles" / "pair_kernel_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(root))
    return csrc, rec


def test_record_matches_only_its_instance(tree):
    _, rec = tree
    assert bench.kernel_traffic_record("mixed", "closed_form", (128, 32)) == 1.4e9
    assert bench.kernel_traffic_record("mixed", "bisect", (128, 32)) is None
    assert bench.kernel_traffic_record("mixed", "closed_form", (64, 8)) is None
    assert bench.kernel_traffic_record("mixed", "closed_form", (128, 32, 16)) is None  # the window instance
    assert bench.kernel_traffic_record("mixed", "closed_form", None) is None  # the default shape (128, 8)
    assert bench.kernel_traffic_record("fp64", "closed_form", (64, 8)) == 2.3e9


def test_record_is_dropped_when_a_source_changes(tree):
    csrc, _ = tree
    with open(csrc / "emppp_api.cu", "a") as fh:
        fh.write("\n")
    assert bench.kernel_traffic_record("mixed", "closed_form", (128, 32)) is None
    assert bench.kernel_traffic_record("fp64", "closed_form", (64, 8)) is None
    assert bench.issue_roofline("mixed", "closed_form", (128, 32), 35.0, {"sm_mhz": 2070.0}, 152) is None


def test_issue_roofline_arithmetic(tree):
    r = bench.issue_roofline("mixed", "closed_form", (128, 32), 40.0, {"sm_mhz": 2000.0}, 150)
    assert r["warp_instructions_per_launch"] == 3.3e10
    assert r["achieved"] == pytest.approx(3.3e10 / 0.040)
    assert r["peak"] == pytest.approx(150 * 4 * 2000e6)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # no clock record: the maximum SM clock
    assert bench.issue_roofline("mixed", "closed_form", (128, 32), 40.0, None, 150)["peak"] == pytest.approx(
        150 * 4 * 2070e6)
    # a record without an instruction count (the FP64 one)
    assert bench.issue_roofline("fp64", "closed_form", (64, 8), 600.0, {"sm_mhz": 2070.0}, 152) is None


def test_committed_record_is_well_formed():
    d = json.load(open(os.path.join(ROOT, "profiles", "pair_kernel_traffic.json")))
    for path in ("mixed", "fp64"):
        e = d[path]
        assert e["dram_bytes_per_launch"] == pytest.approx(e["dram_read_bytes"] + e["dram_write_bytes"])
        assert len(e["sources_sha256_16"]) == 16 and e["command"].startswith("ncu --metrics dram__bytes_read.sum")
        for name in e["sources"]:
            assert os.path.exists(os.path.join(ROOT, "paper_2605_05543_gb300", "csrc", name))


def test_shape_key():
    assert bench.shape_key(None) is None
    t = dict(targets_per_block=128, sources_per_sum=32, history_window=0)
    assert bench.shape_key(t) == (128, 32)
    t["history_window"] = 16
    assert bench.shape_key(t) == (128, 32, 16)
