"""`bench.py --impl reference` (the FP64 oracle as the reference arm) prints
one JSON line with the same metric and workload as the GPU arm, marked as
the reference, with its CPU baseline and an end-to-end figure that moves no
bytes between host and device.  It needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "GLUPS" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["config"]["workload"].startswith("mips_rho1_8192x8192")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_under_torchrun_ranks():
    """Launched as N ranks, rank 0 alone runs the oracle and prints the line;
    the other ranks exit 0 without output."""
    base = dict(os.environ, WORLD_SIZE="2", LOCAL_RANK="0", MASTER_ADDR="127.0.0.1", MASTER_PORT="29555")
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r1 = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=dict(base, RANK="1"))
    assert r1.returncode == 0 and not [ln for ln in r1.stdout.splitlines() if ln.startswith("{")], r1.stdout
    r0 = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=dict(base, RANK="0"))
    assert r0.returncode == 0, r0.stderr[-2000:]
    d = json.loads([ln for ln in r0.stdout.splitlines() if ln.startswith("{")][-1])
    assert d["impl"] == "reference" and d["n_gpus"] == 2


def test_batch_workload_spec_and_oracle_legs():
    """The 256-lattice CIL batch as a benchmark workload: 256 members on the
    rho-bar x activity grid with distinct lattice ids; the oracle legs (the
    reference arm and the CPU baseline) step its centre lattice whole."""
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    wl = bench.workload_spec("batch256")
    ms = wl["members"]
    assert len(ms) == 256 and len({m["lattice_id"] for m in ms}) == 256
    assert wl["nx"] == wl["ny"] == W.CONFIG4["side"]
    assert sorted({m["init"]["rho_mean"] for m in ms}) == sorted(W.CONFIG4["rho_means"])
    assert sorted({m["params"]["B"] for m in ms}) == sorted(W.CONFIG4["activities"])
    assert wl["lattice_id"] == 136 and wl["params"]["B"] == W.CONFIG4["activities"][8]
    rate, steps, dt = bench._oracle_rate(wl, 1024, 1, 0.05)
    assert rate > 0 and steps >= 1
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "batch256", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][0])
    assert d["config"]["workload"] == "cil_rho1_batch256x256x256" and "256x256" in d["config"]["sample"]
