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
    for p in bench.KERNEL_SOURCES:
        os.makedirs(os.path.join(dst, os.path.dirname(p)), exist_ok=True)
        shutil.copy(os.path.join(ROOT, p), os.path.join(dst, p))


def test_kernel_hash_ignores_comments_only(tmp_path, monkeypatch):
    _copy_sources(str(tmp_path))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_hash()
    path = os.path.join(str(tmp_path), bench.KERNEL_SOURCES[0])
    src = open(path).read()
    open(path, "w").write("// an added line comment\n/* and a block\n   comment */\n" + src)
    assert bench.kernel_hash() == h0
    open(path, "w").write(src + "\nnamespace lbm { constexpr int extra_code = 1; }\n")
    assert bench.kernel_hash() != h0


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
            current = entry["kernel_hash"] == bench.kernel_hash()
            assert bench.ncu_traffic(name) == (entry["dram_bytes_per_launch"] if current else None)
