"""The DRAM traffic bench.py reports comes from a committed ncu record keyed
by a hash of the step-kernel sources with comments removed: a comment edit
keeps the record, a code edit voids it (the bench then reports null)."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _copy_sources(dst):
    for p in set(bench.KERNEL_SOURCES[9] + bench.KERNEL_SOURCES[7]):
        os.makedirs(os.path.join(dst, os.path.dirname(p)), exist_ok=True)
        shutil.copy(os.path.join(ROOT, p), os.path.join(dst, p))


def test_kernel_hash_ignores_comments_only(tmp_path, monkeypatch):
    _copy_sources(str(tmp_path))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0, h7 = bench.kernel_hash(9), bench.kernel_hash(7)
    path = os.path.join(str(tmp_path), bench.KERNEL_SOURCES[9][0])
    src = open(path).read()
    open(path, "w").write("// an added line comment\n/* and a block\n   comment */\n" + src)
    assert bench.kernel_hash(9) == h0
    open(path, "w").write(src + "\nnamespace lbm { constexpr int extra_code = 1; }\n")
    assert bench.kernel_hash(9) != h0 and bench.kernel_hash(7) != h7


def test_d2q7_sources_leave_the_d2q9_hash(tmp_path, monkeypatch):
    """A code edit in a D2Q7-only source voids the D2Q7 record, not D2Q9's."""
    _copy_sources(str(tmp_path))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h9, h7 = bench.kernel_hash(9), bench.kernel_hash(7)
    path = os.path.join(str(tmp_path), "paper_1902_00530_gb300/csrc/lbm_step_q7_staged.cuh")
    open(path, "a").write("\nnamespace lbm { constexpr int extra_code7 = 1; }\n")
    assert bench.kernel_hash(9) == h9 and bench.kernel_hash(7) != h7


def test_traffic_record_is_consistent():
    """Each record names an existing capture summary, and the bench reports its
    traffic exactly when the record's hash is that of the current kernels
    (else null: the counters were taken on other code)."""
    import json
    rec = json.load(open(os.path.join(ROOT, "profiles", "step_kernel_traffic.json")))
    for name, entry in rec.items():
        if isinstance(entry, dict):
            assert os.path.exists(os.path.join(ROOT, entry["capture"])), entry["capture"]
            assert entry["dram_bytes_per_launch"] > 0
            current = entry["kernel_hash"] == bench.kernel_hash(entry.get("q", 9))
            assert bench.ncu_traffic(name) == (entry["dram_bytes_per_launch"] if current else None)
