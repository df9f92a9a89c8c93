"""The paper's qualitative results on its own lattice (D2Q7), as GPU smoke
tests: the CIL regime sequence of the increasing-density run of Fig.
Hysteresis (a), and the noise strength at which MIPS stops (App. C.1).  Parameters, box and procedure are the paper's, read from
tests/golden/paper_parameters.json; the regimes are classified with App. D's
cutoffs (paper_1902_00530_gb300.regimes)."""
import json
import os
from collections import Counter

import pytest

import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
G = json.load(open(os.path.join(HERE, "golden", "paper_parameters.json")))


def test_cil_density_sweep_reproduces_paper_regimes():
    """Increasing run at A = 2 (App. C.2-C.3) on the 180 x 60 D2Q7 box, eight
    independent runs in one batch.  At the paper's four snapshot densities
    (HD 0.105, B 0.1425, HO 0.185, RB 0.2875) a majority of the runs is in the
    paper's regime, and the majority regime along the sweep goes HD, B, HO,
    RB and back to HD (the second disordered region at high density, Sec. 4),
    in that order."""
    from paper_1902_00530_gb300 import Lattice, Simulation
    from paper_1902_00530_gb300 import regimes as R
    proc, hyst = G["cil_hysteresis_procedure"], G["cil_hysteresis"]
    d = W.preset("CIL_Q7_PAPER")
    model = d.pop("model")
    nx, ny = G["boxes"]["cil"]
    runs = 8
    sim = Simulation([Lattice(nx, ny, "f32", k, "d2q7") for k in range(runs)], [model] * runs, [d] * runs)
    sim.init(W.seed(11), [dict(W.INIT_PAPER_CIL, rho_mean=proc["rho_start"])] * runs)
    sim.step(proc["init_steps"])
    sweep = R.density_sweep(sim, proc["rho_start"], proc["rho_end"], proc["delta"], proc["t_sample_low"],
                            t_sample_of=lambda r: proc["t_sample_high"] if r > proc["t_switch_rho"] + 1e-9
                            else proc["t_sample_low"], sample=list(range(runs)))
    sim.close()
    majority = []
    for rho, obs in sweep:
        cls = [R.classify_cil(o["phi"], o["drho_y"], o["zeta"], A=d["A"], B=d["B"], rho_bar=rho) for o in obs]
        majority.append((round(rho, 4), Counter(cls).most_common(1)[0][0], cls))
    at = {r: (m, cls) for r, m, cls in majority}
    for regime in ("HD", "B", "HO", "RB"):
        rho = hyst[f"rho_bar_{regime}"]
        m, cls = at[round(rho, 4)]
        assert cls.count(regime) > runs // 2, (rho, regime, cls)
    # order of the stretches of equal majority regime, ignoring one-sample
    # blips where the runs are split at a transition
    stretches = []
    for _, m, _ in majority:
        if stretches and stretches[-1][0] == m:
            stretches[-1][1] += 1
        else:
            stretches.append([m, 1])
    order = []
    for m, n in stretches:
        if n >= 2 and (not order or order[-1] != m):
            order.append(m)
    assert order == ["HD", "B", "HO", "RB", "HD"], stretches


def test_mips_phase_separation_stops_near_paper_sigma():
    """App. C.1 on the 90 x 30 D2Q7 box at rho-bar = 0.12 with Table
    ParametersMIPS (tau = 2): drho (std of rho_y) above the paper's threshold
    0.0430 means phase separated.  Noise strengths 10/700 ... 30/700, three
    realizations each, run side by side as one batch (2 x 10^5 steps, then 50
    samples 4000 steps apart): the mean drho must be above the threshold at
    every sigma below the paper's sigma = 0.0275, where its drho levels out, by
    at least one 1/700 step, and below it at every sigma at least one step
    above.  The liquid and gas densities (20-column windows of rho_y) bracket
    rho-bar in every separated run and approach each other as the noise grows;
    at each sigma the run with the widest gap is taken, since a run that has
    not yet coarsened into one slab has liquid domains narrower than a window."""
    import numpy as np
    from paper_1902_00530_gb300 import Lattice, Simulation
    from paper_1902_00530_gb300 import regimes as R
    ms = G["mips_sweep"]
    d = W.preset("MIPS_Q7_PAPER")
    model = d.pop("model")
    nx, ny = G["boxes"]["mips_phase"]
    sigmas = [k * ms["sigma_step"] for k in range(10, 31, 2)]
    runs = 3
    n = len(sigmas) * runs  # lattice k runs sigmas[k // runs]
    sim = Simulation([Lattice(nx, ny, "f32", k, "d2q7") for k in range(n)], [model] * n,
                     [dict(d, sigma=sigmas[k // runs]) for k in range(n)])
    sim.init(W.seed(12), [dict(W.INIT_CONFIG1, rho_mean=ms["rho_bar"], rho_amp=0.05)] * n)
    sim.step(200_000)
    drho = np.zeros((n, 50))
    for j in range(50):
        sim.step(4000)
        for k in range(n):
            drho[k, j] = sim.observables(k)["drho_y"]
    phases = [R.phase_densities(sim.moments(k)[0]) for k in range(n)]
    sim.close()
    mean = drho.reshape(len(sigmas), runs * 50).mean(1)
    gaps = []
    for a, (s, m) in enumerate(zip(sigmas, mean)):
        if s < ms["sigma_levels_out"] - 2 * ms["sigma_step"]:
            assert R.mips_separated(m), (s, m)
            for liquid, gas in phases[a * runs:(a + 1) * runs]:
                assert gas < ms["rho_bar"] < liquid, (s, liquid, gas)  # App. C.1 phase densities
            gaps.append(max(liquid - gas for liquid, gas in phases[a * runs:(a + 1) * runs]))
        elif s > ms["sigma_levels_out"] + ms["sigma_step"]:
            assert not R.mips_separated(m), (s, m)
    assert gaps[-1] < gaps[0], gaps  # liquid and gas approach each other towards the critical noise


def _cil_up_and_down(runs, seed):
    """phi of every run at every density of the App. C.3 increasing and
    decreasing sweeps, `runs` of each, all in one batch (each lattice on its
    own sampling schedule)."""
    from paper_1902_00530_gb300 import Lattice, Simulation
    from paper_1902_00530_gb300 import regimes as R
    proc = G["cil_hysteresis_procedure"]
    d = W.preset("CIL_Q7_PAPER")
    model = d.pop("model")
    nx, ny = G["boxes"]["cil"]
    up0, down0 = proc["rho_start"], proc["rho_start_down"]
    sim = Simulation([Lattice(nx, ny, "f32", k, "d2q7") for k in range(2 * runs)], [model] * (2 * runs),
                     [d] * (2 * runs))
    sim.init(seed, [dict(W.INIT_PAPER_CIL, rho_mean=up0 if k < runs else down0) for k in range(2 * runs)])
    sim.step(proc["init_steps"])
    ts = lambda r: proc["t_sample_high"] if r > proc["t_switch_rho"] + 1e-9 else proc["t_sample_low"]
    sched = [dict(lattice=k, rho_start=up0, rho_end=proc["rho_end"], delta=proc["delta"], t_sample=ts)
             for k in range(runs)]
    sched += [dict(lattice=runs + k, rho_start=down0, rho_end=up0, delta=-proc["delta"], t_sample=ts)
              for k in range(runs)]
    out = R.density_sweeps(sim, sched)
    sim.close()

    def collect(series):
        by = {}
        for seq in series:
            for r, o in seq:
                by.setdefault(round(r, 4), []).append(o["phi"])
        return by
    return collect(out[:runs]), collect(out[runs:])


def test_cil_hysteresis_loops_at_the_transitions():
    """Fig. Hysteresis (a): increasing and decreasing runs at A = 2 (App. C.3;
    independently initialised), sixteen runs per direction, all 32 in one
    batch with their own sampling schedules.  The mean phi of the two directions must coincide across the
    homogeneous ordered range well inside the paper's B and RB snapshot densities
    (every point within 4.5 standard errors), and must split by more than 5
    standard errors somewhere between the HD and B snapshot densities and
    somewhere above the RB one: the loops at the HD-B transition and at the
    return to disorder at high density."""
    import numpy as np
    hyst = G["cil_hysteresis"]
    up, down = _cil_up_and_down(16, W.seed(21))
    z = {}
    for r in up:
        if r in down:
            a, b = np.array(up[r]), np.array(down[r])
            z[r] = (a.mean() - b.mean()) / max(np.sqrt(a.var() / len(a) + b.var() / len(b)), 1e-12)
    ho = [abs(z[r]) for r in z if hyst["rho_bar_B"] + 0.025 <= r <= hyst["rho_bar_RB"] - 0.04]
    assert len(ho) > 20 and max(ho) < 4.5, max(ho)
    low = [abs(z[r]) for r in z if hyst["rho_bar_HD"] < r < hyst["rho_bar_B"]]
    high = [abs(z[r]) for r in z if r > hyst["rho_bar_RB"]]
    assert max(low) > 5.0, low
    assert max(high) > 5.0, high


def test_cil_phase_diagram_closes_near_paper_critical_point():
    """Fig. PhaseDiagram (App. C.4 procedure: fixed A, rho-bar up by 0.01 every
    10^4 steps), eight runs at each of A = 0, 2, 2.5 and 3 in one batch: the range
    of densities where the majority of runs is ordered (B, HO or RB) narrows
    as A grows and is empty at A = 3, above the paper's critical point
    A_c ~ 2.75, where its four transition lines meet (Sec. 5); at A = 2.5 the
    homogeneous ordered window still holds the paper's rho-bar_c ~ 0.18.
    Above B - A rho-bar^2 = 0 every run is classified motionless.  At A = 0 the
    model is a plain polar active fluid (Sec. 5): B and HO appear, RB does not."""
    from paper_1902_00530_gb300 import Lattice, Simulation
    from paper_1902_00530_gb300 import regimes as R
    pd, proc = G["cil_phase_diagram"], G["cil_hysteresis_procedure"]
    d0 = W.preset("CIL_Q7_PAPER")
    model = d0.pop("model")
    nx, ny = G["boxes"]["cil"]
    As, runs = (0.0, 2.0, 2.5, 3.0), 8
    lats = [Lattice(nx, ny, "f32", a * runs + r, "d2q7") for a in range(len(As)) for r in range(runs)]
    prms = [dict(d0, A=A) for A in As for _ in range(runs)]
    sim = Simulation(lats, [model] * len(lats), prms)
    sim.init(W.seed(31), [dict(W.INIT_PAPER_CIL, rho_mean=proc["rho_start"])] * len(lats))
    sim.step(proc["init_steps"])
    sched = [dict(lattice=k, rho_start=proc["rho_start"], rho_end=proc["rho_end"], delta=pd["delta"],
                  t_sample=pd["t_sample"]) for k in range(len(lats))]
    out = R.density_sweeps(sim, sched)
    sim.close()
    ordered, ho, majority = {}, {}, {}
    for a, A in enumerate(As):
        ordered[A], ho[A], majority[A] = [], [], []
        for j in range(len(out[0])):
            rho = out[a * runs][j][0]
            cls = [R.classify_cil(o["phi"], o["drho_y"], o["zeta"], A=A, B=d0["B"], rho_bar=rho)
                   for o in (out[a * runs + r][j][1] for r in range(runs))]
            top, n = Counter(cls).most_common(1)[0]
            majority[A].append(top if n > runs // 2 else None)
            if 0.3 - A * rho * rho <= 0:
                assert cls == ["motionless"] * runs, (A, rho, cls)
            if n > runs // 2 and top in ("B", "HO", "RB"):
                ordered[A].append(rho)
            if n > runs // 2 and top == "HO":
                ho[A].append(rho)
    assert len(ordered[2.0]) > len(ordered[2.5]) > 0 and ordered[3.0] == [], ordered
    assert min(ho[2.5]) - 1e-9 <= pd["rho_bar_c"] <= max(ho[2.5]) + 1e-9, ho[2.5]
    # A = 0 (Sec. 5): a Vicsek-like polar fluid, HD -> B -> HO, no reverse banding
    assert "B" in majority[0.0] and "HO" in majority[0.0] and "RB" not in majority[0.0], majority[0.0]
