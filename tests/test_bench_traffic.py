"""The bench's recorded DRAM traffic: a record stays valid while the kernel's code is unchanged (comments and
blank lines do not count) and is voided by any change of the code."""
import json
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _copy_tree(tmp_path):
    csrc = tmp_path / "paper_2405_12913_gb300" / "csrc"
    shutil.copytree(os.path.join(ROOT, "paper_2405_12913_gb300", "csrc"), csrc)
    (tmp_path / "profiles").mkdir()
    return csrc


def test_the_hash_ignores_comments_and_blank_lines_but_not_code(tmp_path, monkeypatch):
    csrc = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash("kick_drift")
    f = csrc / "mesh_kernels.cu"
    text = f.read_text()
    f.write_text("// a new comment line\n\n" + text.replace("\n", "  \n", 3) + "\n/* a block\n comment */\n")
    assert bench.kernel_source_hash("kick_drift") == h0
    f.write_text(text.replace("kick_drift_kernel", "kick_drift_kernel_", 1))
    assert bench.kernel_source_hash("kick_drift") != h0


def test_a_record_is_used_only_with_its_hash(tmp_path, monkeypatch):
    _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_source_hash("kspace")
    rec = {"w": {"kspace": {"dram_bytes_per_launch": 123, "source_hash": h}}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("kspace", "w") == 123
    assert bench.recorded_traffic("kspace", "other workload") is None
    rec["w"]["kspace"]["source_hash"] = "0" * 16
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("kspace", "w") is None


def test_the_committed_records_match_the_committed_kernels():
    # every record in profiles/traffic.json was taken on the kernels as they stand
    recs = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for workload, kernels in recs.items():
        for kernel, rec in kernels.items():
            assert rec["source_hash"] == bench.kernel_source_hash(kernel), (workload, kernel)
