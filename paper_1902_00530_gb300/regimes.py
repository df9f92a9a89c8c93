"""Regime classification and adiabatic sweeps (App. C and D of arXiv:1902.00530).

Host-side logic on top of the observables the library reduces on the GPU:

* ``classify_cil``: the App. D table for the CIL model -- homogeneous
  disordered (HD: phi below its cutoff), homogeneous ordered (HO: drho at or
  below its cutoff), banding (B) and reverse banding (RB: zeta above its
  cutoff), plus "motionless" where B - A rho-bar^2 <= 0 (the paper's fifth,
  trivial phase).
* ``mips_separated``: App. C.1's phase-separation criterion drho > 0.0430.
* ``density_sweep``: App. C.3's adiabatic procedure -- step t_sample steps,
  take a sample, change the mean density by delta (App. C.2), repeat.
* ``density_sweeps``: several such sweeps with their own schedules (start,
  end, step, sampling interval) on the lattices of one batch -- the paper's
  increasing and decreasing runs side by side.
* ``phase_densities``: App. C.1's liquid and gas densities of a phase-separated
  state -- the column profile rho_y(x) averaged over a window 20 columns wide,
  slid along the periodic box; the highest window is the liquid, the lowest
  the gas.

The paper's cutoffs are in its units (mean densities 0.1-0.35).  Under the
model's density-rescaling symmetry (rho -> s rho with C/s, s rho*, A/s^2,
s sigma) velocities are unchanged and densities scale by s, so phi and zeta
cutoffs carry over while the drho cutoffs scale by s: pass
``density_scale = s`` for the rescaled ("RHO1") presets.
"""
from __future__ import annotations

PHI_CUT = 0.024           # App. D: phi < 0.024 is HD (CIL)
DRHO_CUT_CIL = 0.012      # App. D: drho > 0.012 is B or RB
ZETA_CUT = 0.1            # App. D: zeta > 0.1 is RB
DRHO_CUT_MIPS = 0.0430    # App. C.1: drho > 0.0430 is phase separated
PHASE_WINDOW = 20         # App. C.1: the averaging window is 20 dx wide


def classify_cil(phi: float, drho: float, zeta: float, density_scale: float = 1.0,
                 A: float | None = None, B: float | None = None, rho_bar: float | None = None) -> str:
    """The App. D regime of one CIL sample (or of averaged observables)."""
    if A is not None and B is not None and rho_bar is not None and B - A * rho_bar * rho_bar <= 0:
        return "motionless"
    if phi < PHI_CUT:
        return "HD"
    if drho <= DRHO_CUT_CIL * density_scale:
        return "HO"
    return "RB" if zeta > ZETA_CUT else "B"


def mips_separated(drho: float, density_scale: float = 1.0) -> bool:
    """App. C.1: phase separation when drho exceeds 0.0430 (paper units)."""
    return drho > DRHO_CUT_MIPS * density_scale


def density_sweep(sim, rho_start: float, rho_end: float, delta: float, t_sample: int, lattice: int = -1,
                  t_sample_of=None, sample=None):
    """App. C.3: from mean density rho_start, repeat {step t_sample steps; sample
    the observables; add delta to the mean density} until rho_end is passed.
    ``t_sample_of(rho)`` may vary the interval with the density (the paper uses
    500 steps above rho-bar 0.2 and 1500 below).  ``lattice`` is the lattice
    whose density changes (-1: all).  Returns [(rho_bar, obs)] with obs the
    record of lattice ``sample`` if that is an int, a list of records if it is
    a sequence of lattices (the paper's repeated runs, as one batch), and of
    ``lattice`` (0 if -1) by default."""
    if delta == 0 or (rho_end - rho_start) * delta < 0:
        raise ValueError("delta must move rho_start towards rho_end")
    out = []
    rho = rho_start
    k = 0
    if sample is None:
        sample = lattice if lattice >= 0 else 0
    while (rho - rho_end) * (1 if delta > 0 else -1) <= 1e-12:
        sim.step(t_sample_of(rho) if t_sample_of else t_sample)
        if isinstance(sample, int):
            out.append((rho, sim.observables(sample)))
        else:
            out.append((rho, [sim.observables(k_) for k_ in sample]))
        sim.add_density(delta, lattice)
        k += 1
        rho = rho_start + k * delta
    return out


def density_sweeps(sim, schedules):
    """App. C.3 sweeps of several lattices of one batch, each with its own
    schedule: a dict with `lattice`, `rho_start`, `rho_end`, `delta` and
    `t_sample` (steps, or a function of the current mean density).  Every
    lattice keeps its own countdown; the batch is stepped to the next due
    sample, the due lattices are sampled (just before their density change,
    as in App. C.3) and shifted by their delta.  A lattice whose sweep is over
    keeps being stepped with the others.  Returns, per schedule, the list of
    (rho_bar, observables)."""
    state = []
    for sch in schedules:
        if sch["delta"] == 0 or (sch["rho_end"] - sch["rho_start"]) * sch["delta"] < 0:
            raise ValueError("delta must move rho_start towards rho_end")
        ts = sch["t_sample"]
        interval = ts if callable(ts) else (lambda r, ts=ts: ts)
        state.append(dict(sch=sch, interval=interval, k=0, rho=sch["rho_start"], out=[],
                          left=int(interval(sch["rho_start"]))))

    def active(st):
        sch = st["sch"]
        return (st["rho"] - sch["rho_end"]) * (1 if sch["delta"] > 0 else -1) <= 1e-12

    while any(active(st) for st in state):
        n = min(st["left"] for st in state if active(st))
        sim.step(n)
        for st in state:
            if not active(st):
                continue
            st["left"] -= n
            if st["left"] == 0:
                sch = st["sch"]
                st["out"].append((st["rho"], sim.observables(sch["lattice"])))
                sim.add_density(sch["delta"], sch["lattice"])
                st["k"] += 1
                st["rho"] = sch["rho_start"] + st["k"] * sch["delta"]
                if active(st):
                    st["left"] = int(st["interval"](st["rho"]))
    return [st["out"] for st in state]


def phase_densities(rho, width: int = PHASE_WINDOW):
    """App. C.1: (liquid, gas) densities of a phase-separated state from its
    density field rho (ny, nx) -- or from its column profile rho_y(x) -- by
    averaging rho_y over `width` consecutive columns (periodic) at every
    offset and taking the highest and the lowest window.  Accepts numpy
    arrays and (CPU or CUDA) torch tensors."""
    import numpy as np
    if hasattr(rho, "detach"):
        rho = rho.detach().double().cpu().numpy()
    a = np.asarray(rho, dtype=np.float64)
    prof = a.mean(axis=0) if a.ndim == 2 else a
    nx = prof.shape[0]
    if not 1 <= width <= nx:
        raise ValueError("window width must be in [1, nx]")
    ext = np.concatenate([prof, prof[:width - 1]])
    c = np.concatenate([[0.0], np.cumsum(ext)])
    windows = (c[width:width + nx] - c[:nx]) / width
    return float(windows.max()), float(windows.min())
