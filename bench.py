"""Throughput of the fused active-LBM step on GB300.

Default workload: the 8192 x 8192 periodic D2Q9 lattice with the rescaled MIPS
closure (grad-rho gradient, noise, negative correction), FP32 populations,
observables sampled every 100 steps -- the precision/throughput configuration
whose roofline target is stated for an 8192^2 lattice.  One "step" is one
update of every site (all steps of the method).  Inputs (4.8 GB of populations)
exceed the 129 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank advances its own
independent lattice (replicas: the method has no exchange between lattices).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLUPS & % HBM roofline; batched/16-bit-storage vs plain FP32 at stated error"
UNIT = "GLUPS"
BYTES_PER_UPDATE = {"f32": 72, "f16s": 36, "bf16s": 36}   # 9 reads + 9 writes per site


def bytes_per_update(storage: str, q: int = 9) -> int:
    """Algorithmic HBM bytes of one site update: q populations read and written."""
    return BYTES_PER_UPDATE[storage] * q // 9
# The sources each velocity set's step kernels are compiled from (the D2Q7
# kernels include the D2Q9 headers).
KERNEL_SOURCES = {
    9: ["paper_1902_00530_gb300/csrc/lbm_device.cuh", "paper_1902_00530_gb300/csrc/lbm_step.cuh",
        "paper_1902_00530_gb300/csrc/lbm_step_staged.cuh"],
    7: ["paper_1902_00530_gb300/csrc/lbm_device.cuh", "paper_1902_00530_gb300/csrc/lbm_step.cuh",
        "paper_1902_00530_gb300/csrc/lbm_step_staged.cuh", "paper_1902_00530_gb300/csrc/lbm_step_q7.cuh",
        "paper_1902_00530_gb300/csrc/lbm_step_q7_staged.cuh"],
}


def kernel_hash(q: int = 9) -> str:
    """Hash of the velocity set's step-kernel sources with comments removed and
    whitespace collapsed: the recorded DRAM traffic stays valid across comment
    and layout edits, not across code changes."""
    h = hashlib.sha256()
    for p in KERNEL_SOURCES[q]:
        with open(os.path.join(ROOT, p), encoding="utf-8") as f:
            code = re.sub(r"/\*.*?\*/", " ", f.read(), flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ncu_traffic(workload: str):
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    if it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    entry = rec.get(workload)
    if not entry or entry.get("kernel_hash") != kernel_hash(entry.get("q", 9)):
        return None
    return entry.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank: int):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        self.gpu = ids[local_rank] if local_rank < len(ids) else str(local_rank)
        self.proc = None
        self.t_begin = self.t_end = None
        self.out = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def mark_begin(self):
        self.t_begin = time.time()

    def mark_end(self):
        self.t_end = time.time()

    def stop(self) -> dict:
        import datetime
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.flush()
        self.out.seek(0)
        rows = [r.strip().split(", ") for r in self.out.read().strip().splitlines() if r.strip()]
        os.unlink(self.out.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(r[0].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            if ts is not None and self.t_begin is not None and not (self.t_begin - 0.05 <= ts <= self.t_end + 0.05):
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate_over_ranks(cells_per_rank: int, steps: int, ms_local: float, world: int, dist=None):
    """Replicas: every rank advances its own lattice (lattice id = rank), so the
    whole-job rate is the work of all ranks over the slowest rank's time."""
    ms = ms_local
    if world > 1 and dist is not None:
        import torch
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([ms_local], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * cells_per_rank * steps / (ms * 1e-3) / 1e9, ms


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload_spec(name: str):
    import workloads as W
    if name == "mips8192":
        d = W.preset("MIPS_RHO1")
        return dict(nx=8192, ny=8192, model=d.pop("model"), params=d, init=W.INIT_CONFIG1, sample_every=100,
                    seed=W.seed(3), label="mips_rho1_8192x8192")
    if name == "mips4096":  # a smaller case of the same workload, for profiler captures
        d = W.preset("MIPS_RHO1")
        return dict(nx=4096, ny=4096, model=d.pop("model"), params=d, init=W.INIT_CONFIG1, sample_every=100,
                    seed=W.seed(3), label="mips_rho1_4096x4096")
    if name == "cil8192":  # the CIL closure at the benchmark's size (FP32 copy-bound with noise)
        d = W.preset("CIL_RHO1")
        return dict(nx=8192, ny=8192, model=d.pop("model"), params=d, init=W.INIT_CONFIG2, sample_every=100,
                    seed=W.seed(3), label="cil_rho1_8192x8192")
    if name == "cil1024":
        d = W.preset("CIL_RHO1")
        return dict(nx=1024, ny=1024, model=d.pop("model"), params=d, init=W.INIT_CONFIG2, sample_every=100,
                    seed=W.seed(2), label="cil_rho1_1024x1024")
    if name == "batch256":  # 256 CIL lattices of 256^2 on the rho-bar x activity grid, one launch per step
        c4 = W.CONFIG4
        d = W.preset(c4["preset"])
        model = d.pop("model")
        members = [dict(params=dict(d, B=act), init=dict(c4["init"], rho_mean=rm), lattice_id=i * 16 + j)
                   for i, rm in enumerate(c4["rho_means"]) for j, act in enumerate(c4["activities"])]
        mid = members[8 * 16 + 8]  # the grid's centre: the lattice the oracle legs step
        return dict(nx=c4["side"], ny=c4["side"], model=model, params=mid["params"], init=mid["init"],
                    lattice_id=mid["lattice_id"], sample_every=100, seed=W.seed(4),
                    label="cil_rho1_batch256x256x256", members=members)
    if name in ("mips7_8192", "mips7_4096"):  # the paper's D2Q7 lattice, same physics and sizes
        n = 8192 if name == "mips7_8192" else 4096
        d = W.preset("MIPS_Q7_RHO1")
        return dict(nx=n, ny=n, model=d.pop("model"), params=d, init=W.INIT_CONFIG1, sample_every=100,
                    seed=W.seed(3), label=f"mips_q7_rho1_{n}x{n}", velocity_set="d2q7")
    raise SystemExit(f"unknown workload {name}")


def run_gpu(args, world, rank, local):
    import torch
    import torch.distributed as dist
    from paper_1902_00530_gb300 import Lattice, Simulation

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wl = workload_spec(args.workload)
    storage = args.storage
    vs = wl.get("velocity_set", "d2q9")
    q = 7 if vs == "d2q7" else 9
    members = wl.get("members") or [dict(params=wl["params"], init=wl["init"], lattice_id=0)]
    nlat = len(members)
    # replicas (one per rank) take disjoint lattice ids
    lats = [Lattice(wl["nx"], wl["ny"], storage, rank * nlat + m["lattice_id"], vs) for m in members]
    sim = Simulation(lats, [wl["model"]] * nlat, [m["params"] for m in members],
                     sample_every=wl["sample_every"], ring_capacity=max(16, args.steps // wl["sample_every"] + 4))
    sim.init(wl["seed"], [m["init"] for m in members])
    sim.set_persistent({"auto": 2, "on": 1, "off": 0}[args.persistent])
    if args.shape:
        sh = [int(x) for x in args.shape.split(",")]
        sim.set_tuning(1, *sh)
    else:
        sim.tune()
    shape = sim.get_tuning()
    persistent = sim.get_persistent()
    sim.step(args.warmup)
    sim.synchronize()
    cells = wl["nx"] * wl["ny"] * nlat

    # ---------------- timed region: K steps, events on the library's stream --
    sim.set_profiling(True)
    sim.profile_read()
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)  # let the sampler start before the work
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler.mark_begin()
    e0.record(sim.stream)
    sim.step(args.steps)
    launches = sim.last_launch_count()
    e1.record(sim.stream)
    e1.synchronize()
    torch.cuda.synchronize()
    sampler.mark_end()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    prof = sim.profile_read()
    sim.set_profiling(False)
    ms = e0.elapsed_time(e1)
    value, ms_max = aggregate_over_ranks(cells, args.steps, ms, world, dist if world > 1 else None)

    # ---------------- roofline of the dominant kernel (the fused step) -------
    peak, peak_kind = measured_peak()
    step_avg_ms = prof["step_ms"] / max(prof["step_launches"], 1)
    achieved = bytes_per_update(storage, q) * cells / (step_avg_ms * 1e-3) / 1e9
    traffic = ncu_traffic(f"{wl['label']}_{storage}")
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": bytes_per_update(storage, q) * cells,
                "kernel": "lbm::step_persistent_kernel" if persistent and shape[3] == 0 else
                          ("lbm::step_staged_kernel" if shape[3] > 0 else "lbm::step_kernel") +
                          ("_q7" if q == 7 else ""), "avg_launch_ms": round(step_avg_ms, 5),
                "step_kernel_share": round(prof["step_ms"] / max(prof["step_ms"] + prof["other_ms"], 1e-9), 4),
                "frac_of_8TBps": round(achieved / 8000.0, 4)}

    # ---------------- end to end through the C ABI with host buffers ---------
    host_state = [sim.get_state(k, host=True) for k in range(nlat)]  # pinned inputs, outside the timed region
    out_state = [torch.empty_like(h).pin_memory() for h in host_state]
    state_bytes = sum(h.numel() for h in host_state) * 4
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(nlat):
        sim.set_state(host_state[k], k)    # H2D of the populations (returns when the copy is done)
    t_h2d = time.perf_counter()
    sim.step(args.steps)
    sim.synchronize()
    t_d2h = time.perf_counter()
    for k in range(nlat):
        sim.get_state(k, host=True, out=out_state[k])  # D2H of the result
    t_d2h_end = time.perf_counter()
    obs = sim.observables()                # D2H of the observables (syncs)
    t1 = time.perf_counter()
    e2e_value, _ = aggregate_over_ranks(cells, args.steps, (t1 - t0) * 1e3, world, dist if world > 1 else None)
    e2e = {"value": round(e2e_value, 3), "unit": UNIT,
           "h2d_bytes_per_step": round(state_bytes / args.steps, 1),
           "d2h_bytes_per_step": round((state_bytes + 56) / args.steps, 1),
           "h2d_gbs": round(state_bytes / (t_h2d - t0) / 1e9, 1),
           "d2h_gbs": round(state_bytes / (t_d2h_end - t_d2h) / 1e9, 1),
           "note": "one upload of the populations, the K steps, one download and the observables: "
                   "the copies are spread over K steps"}
    del out_state, host_state
    sim.close()
    del sim
    torch.cuda.empty_cache()

    extra = {}
    if rank == 0 and not args.quick:
        extra = secondary_lines(args, wl)
    return dict(value=value, ms=ms_max, clocks=clocks, roofline=roofline, e2e=e2e, launches=launches,
                obs=obs, extra=extra, wl=wl, shape=shape, persistent=persistent, cells=cells, nlat=nlat, q=q)


def secondary_lines(args, wl):
    """The metric's comparison forms on the same GPU: 16-bit shifted storage of
    the same workload, and the batched forms (256 lattices of 256^2 CIL on a
    density x activity grid; a ragged mixed-model batch)."""
    import torch
    import workloads as W
    from paper_1902_00530_gb300 import Lattice, Simulation
    out = {}
    steps = max(50, min(args.steps, 300))

    def time_sim(sim, cells, steps):
        sim.tune()
        sim.step(5)
        sim.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(sim.stream)
        sim.step(steps)
        e1.record(sim.stream)
        e1.synchronize()
        return cells * steps / (e0.elapsed_time(e1) * 1e-3) / 1e9

    for st in ("f16s", "bf16s"):
        sim = Simulation([Lattice(wl["nx"], wl["ny"], st, 0, wl.get("velocity_set", "d2q9"))], [wl["model"]],
                         [wl["params"]],
                         sample_every=wl["sample_every"], ring_capacity=16)
        sim.init(wl["seed"], [wl["init"]])
        out[f"{st}_glups"] = round(time_sim(sim, wl["nx"] * wl["ny"], steps), 2)
        sim.close()
        del sim
        torch.cuda.empty_cache()
    # the CIL closure at the same size, where FP32 storage runs at the copy
    # bandwidth: the case 16-bit storage is for
    if wl.get("velocity_set", "d2q9") == "d2q9" and wl["nx"] == 8192:
        wc = workload_spec("cil8192")
        peak, _ = measured_peak()
        for st in ("f32", "f16s", "bf16s"):
            sim = Simulation([Lattice(wc["nx"], wc["ny"], st)], [wc["model"]], [wc["params"]],
                             sample_every=wc["sample_every"], ring_capacity=16)
            sim.init(wc["seed"], [wc["init"]])
            g = time_sim(sim, wc["nx"] * wc["ny"], steps)
            out[f"cil8192_{st}_glups"] = round(g, 2)
            out[f"cil8192_{st}_frac_hbm"] = round(g * bytes_per_update(st) / peak, 4)
            sim.close()
            del sim
            torch.cuda.empty_cache()
    # uniform batch: 256 CIL lattices of 256^2, rho-bar x activity (B) grid
    c4 = W.CONFIG4
    d = W.preset(c4["preset"])
    model = d.pop("model")
    for st in ("f32", "f16s"):
        lats, prms, specs = [], [], []
        for i, rm in enumerate(c4["rho_means"]):
            for j, act in enumerate(c4["activities"]):
                lats.append(Lattice(c4["side"], c4["side"], st, i * 16 + j))
                prms.append(dict(d, B=act))
                specs.append(dict(c4["init"], rho_mean=rm))
        sim = Simulation(lats, [model] * len(lats), prms, sample_every=100, ring_capacity=16)
        sim.init(W.seed(4), specs)
        out[f"batch256_cil_{st}_glups"] = round(time_sim(sim, len(lats) * c4["side"] ** 2, steps), 2)
        sim.close()
        del sim
        torch.cuda.empty_cache()
    # ragged batch: 64 lattices, sides from {128..2048}, mixed MIPS/CIL (two
    # launch groups, run as parallel graph branches)
    rag = W.ragged_batch()
    for st in ("bf16s", "f16s", "f32"):
        lats, mods, prms, specs = [], [], [], []
        for k, (side, pname) in enumerate(rag):
            dd = W.preset(pname)
            mods.append(dd.pop("model"))
            prms.append(dd)
            lats.append(Lattice(side, side, st, k))
            specs.append(W.INIT_CONFIG1 if mods[-1] == "mips" else W.INIT_CONFIG2)
        sim = Simulation(lats, mods, prms, sample_every=100, ring_capacity=16)
        sim.init(W.seed(5), specs)
        out[f"ragged64_{st}_glups"] = round(time_sim(sim, sum(s * s for s, _ in rag), steps), 2)
        sim.close()
        del sim
        torch.cuda.empty_cache()
    # the paper's own lattice: D2Q7 at the same size and physics (56 B per FP32 update)
    if wl.get("velocity_set", "d2q9") == "d2q9" and wl["nx"] == 8192:
        w7 = workload_spec("mips7_8192")
        peak, _ = measured_peak()
        for st in ("f32", "bf16s"):
            sim = Simulation([Lattice(w7["nx"], w7["ny"], st, 0, "d2q7")], [w7["model"]], [w7["params"]],
                             sample_every=w7["sample_every"], ring_capacity=16)
            sim.init(w7["seed"], [w7["init"]])
            g = time_sim(sim, w7["nx"] * w7["ny"], steps)
            out[f"d2q7_mips_8192_{st}_glups"] = round(g, 2)
            out[f"d2q7_mips_8192_{st}_frac_hbm"] = round(g * bytes_per_update(st, 7) / peak, 4)
            sim.close()
            del sim
            torch.cuda.empty_cache()
    return out


def _oracle_pair(wl):
    """The oracle's (init, run) for the workload's lattice."""
    import oracle as O
    return (O.init7, O.run7) if wl.get("velocity_set") == "d2q7" else (O.init, O.run)


def _oracle_rate(wl, n: int, threads: int, budget_s: float):
    """Site updates per second of the FP64 oracle, as it stands, stepping an
    n x n window of the workload (same seed, parameters and global
    coordinates) until about budget_s seconds have passed."""
    import oracle as O
    init, run = _oracle_pair(wl)
    p = O.params(**wl["params"])
    n = min(n, wl["nx"], wl["ny"])  # a batch's lattice: the whole (periodic) lattice
    win = (0, 0, wl["nx"], wl["ny"])
    lid = wl.get("lattice_id", 0)
    f = init(n, n, wl["seed"], lattice_id=lid, **wl["init"], prm=p, window=win)
    f = run(f, wl["model"], p, wl["seed"], 0, 1, lattice_id=lid, window=win, threads=threads)  # load, warm
    steps, t0 = 1, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        f = run(f, wl["model"], p, wl["seed"], steps, 2, lattice_id=lid, window=win, threads=threads)
        steps += 2
    dt = time.perf_counter() - t0
    return n * n * (steps - 1) / dt, steps - 1, dt


def cpu_baseline(wl, budget_s: float = 10.0):
    """The FP64 oracle on the host: single-threaded on a 512^2 window, and on
    all host cores (OpenMP over rows, the same arithmetic) on a 1024^2 window
    of the same workload.  The line's value is the all-cores figure."""
    import oracle as O
    r1, s1, t1 = _oracle_rate(wl, 512, 1, budget_s)
    cores = O.host_cores()
    used = O.threads_in_use(cores)
    rn, sn, tn = _oracle_rate(wl, 1024, used, budget_s)
    nn, n1 = min(1024, wl["nx"], wl["ny"]), min(512, wl["nx"], wl["ny"])
    return {"value": round(rn / 1e9, 6), "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"{nn}x{nn} window of the {wl['label']} workload, {sn} steps, FP64, {used} threads, "
                      f"{tn:.1f} s",
            "single_thread": {"value": round(r1 / 1e9, 6), "unit": UNIT, "cores": 1,
                              "sample": f"{n1}x{n1} window, {s1} steps, FP64, 1 thread, {t1:.1f} s"},
            "host_cores": cores}


def run_reference(args, world, rank):
    """The oracle as the reference arm: each step advances an n x n window of
    the workload by one step on all host cores (OpenMP over rows; n = 1024,
    smaller for long runs so the whole run stays within a few minutes)."""
    if rank != 0:
        return
    import oracle as O
    wl = workload_spec(args.workload)
    cores = O.host_cores()
    threads = O.threads_in_use(cores)
    n = min(1024, wl["nx"], wl["ny"])
    while n > 64 and n * n * (args.steps + args.warmup) > 2.0e7 * max(threads, 1):
        n //= 2
    init, run = _oracle_pair(wl)
    p = O.params(**wl["params"])
    win = (0, 0, wl["nx"], wl["ny"])
    lid = wl.get("lattice_id", 0)
    f = init(n, n, wl["seed"], lattice_id=lid, **wl["init"], prm=p, window=win)
    f = run(f, wl["model"], p, wl["seed"], 0, args.warmup, lattice_id=lid, window=win, threads=threads)
    t0 = time.perf_counter()
    f = run(f, wl["model"], p, wl["seed"], args.warmup, args.steps, lattice_id=lid, window=win, threads=threads)
    dt = time.perf_counter() - t0
    value = n * n * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)",
            "config": {"workload": wl["label"],
                       "sample": f"{n}x{n} window per step, FP64 oracle, {threads} threads"},
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{n}x{n} window of {wl['label']}, {args.steps} steps, "
                                       f"{threads} threads ({cores} host cores)"},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mips8192")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16s", "bf16s"])
    ap.add_argument("--quick", action="store_true", help="skip the secondary (16-bit, batched) lines")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shape", default="", help="fixed launch shape vec,rows,warps[,stages] instead of tuning")
    ap.add_argument("--persistent", default="auto", choices=["auto", "on", "off"],
                    help="persistent launches of the direct kernel: chosen by the tuner (default), always, never")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    r = run_gpu(args, world, rank, local)
    if rank != 0:
        return
    base = None if args.no_cpu_baseline or world > 1 else cpu_baseline(r["wl"])
    clocks = r["clocks"]
    wl = r["wl"]
    pop_bytes = r["cells"] * r["q"] * (4 if args.storage == "f32" else 2)
    line = {
        "metric": METRIC, "value": round(r["value"], 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(r["ms"] / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.storage == "f32" else args.storage,
        "data": "synthetic (seeded lattice, paper-shaped parameters)",
        "config": {"workload": wl["label"] + "_" + args.storage, "nx": wl["nx"], "ny": wl["ny"],
                   "lattices": r["nlat"],
                   "closure": wl["model"], "storage": args.storage, "sample_every": wl["sample_every"],
                   "replicas": world,
                   "l2": f"inputs larger than L2 (populations {2 * pop_bytes / 1e9:.1f} GB, both buffers, "
                         f"against 0.13 GB of L2); no flush" if 2 * pop_bytes > 129e6 else
                         "inputs fit L2: effective, not HBM, rates",
                   "timing": "CUDA events on the library stream around lbm_step(K); per-kernel event pairs",
                   "launch_shape": {"vec": r["shape"][0], "rows": r["shape"][1], "warps": r["shape"][2],
                                    "stages": r["shape"][3],
                                    "kernel": "staged (bulk-copy rows in shared memory)" if r["shape"][3]
                                    else "persistent (direct-kernel steps, one launch per stretch of steps "
                                         "between samples)" if r["persistent"]
                                    else "direct (vector loads + shuffles)",
                                    "chosen_by": "fixed" if args.shape else "tuner"}},
        "gpu_launches": r["launches"],
        "clocks": clocks,
        "roofline": r["roofline"],
        "e2e": r["e2e"],
        "cpu_baseline": base,
        "secondary": r["extra"],
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
