"""App. D regime table and the App. C.3 sweep loop (host logic, no GPU)."""
import json
import os

import pytest

from paper_1902_00530_gb300 import regimes as R

HERE = os.path.dirname(os.path.abspath(__file__))
G = json.load(open(os.path.join(HERE, "golden", "paper_parameters.json")))


def test_cutoffs_are_the_papers():
    assert R.PHI_CUT == G["cil_thresholds"]["phi"]
    assert R.DRHO_CUT_CIL == G["cil_thresholds"]["drho"]
    assert R.ZETA_CUT == G["cil_thresholds"]["zeta"]
    assert R.DRHO_CUT_MIPS == G["mips_sweep"]["drho_threshold"]


@pytest.mark.parametrize("phi,drho,zeta,expect", [
    (0.010, 0.050, 0.20, "HD"),      # phi below cutoff: HD whatever the rest
    (0.024, 0.012, 0.20, "HO"),      # at both cutoffs: ordered, homogeneous
    (0.100, 0.013, 0.05, "B"),
    (0.100, 0.013, 0.10, "B"),       # zeta at the cutoff is not RB
    (0.100, 0.030, 0.15, "RB"),
])
def test_cil_table(phi, drho, zeta, expect):
    assert R.classify_cil(phi, drho, zeta) == expect


def test_density_scale_moves_only_drho_cutoff():
    s = 1 / 0.185
    assert R.classify_cil(0.1, 0.012 * s * 0.99, 0.2, density_scale=s) == "HO"
    assert R.classify_cil(0.1, 0.012 * s * 1.01, 0.2, density_scale=s) == "RB"
    assert R.classify_cil(0.0239, 1.0, 1.0, density_scale=s) == "HD"
    assert R.mips_separated(0.0431) and not R.mips_separated(0.0429)
    assert R.mips_separated(0.0431 / 0.12, density_scale=1 / 0.12)


def test_motionless_above_the_U0_line():
    # App. D: B - A rho-bar^2 <= 0 is the trivial no-motion phase
    assert R.classify_cil(0.2, 0.0, 0.0, A=2.0, B=0.3, rho_bar=0.39) == "motionless"
    assert R.classify_cil(0.2, 0.0, 0.0, A=2.0, B=0.3, rho_bar=0.38) == "HO"


class FakeSim:
    def __init__(self):
        self.log = []
        self.rho = 0.09

    def step(self, n):
        self.log.append(("step", n))

    def observables(self, lattice=0):
        return {"rho": self.rho, "lattice": lattice}

    def add_density(self, delta, lattice=-1):
        self.rho += delta
        self.log.append(("add", round(delta, 6)))


def test_density_sweep_follows_app_c3():
    sim = FakeSim()
    res = R.density_sweep(sim, 0.09, 0.1, 0.0025, 1500,
                          t_sample_of=lambda r: 500 if r > 0.2 else 1500)
    assert [round(r, 6) for r, _ in res] == [0.09, 0.0925, 0.095, 0.0975, 0.1]
    assert sim.log[0] == ("step", 1500) and sim.log[1] == ("add", 0.0025)
    sim = FakeSim()
    down = R.density_sweep(sim, 0.35, 0.345, -0.0025, 500)
    assert [round(r, 6) for r, _ in down] == [0.35, 0.3475, 0.345]
    with pytest.raises(ValueError):
        R.density_sweep(sim, 0.1, 0.2, -0.01, 10)


def test_density_sweep_samples_a_batch():
    sim = FakeSim()
    res = R.density_sweep(sim, 0.09, 0.095, 0.0025, 100, sample=[0, 1, 2])
    assert len(res) == 3 and [o["lattice"] for o in res[0][1]] == [0, 1, 2]
    assert res[1][1][2]["rho"] == pytest.approx(0.0925)


def test_phase_densities_window():
    """App. C.1: a liquid strip of 40 columns at 0.19 in a 0.05 gas, crossing
    the periodic edge: the 20-column windows find both densities exactly; a
    smooth profile matches a brute-force loop over window offsets."""
    import numpy as np
    nx, ny = 90, 30
    prof = np.full(nx, 0.05)
    prof[np.r_[70:90, 0:20]] = 0.19
    rho = np.tile(prof, (ny, 1))
    liq, gas = R.phase_densities(rho)
    assert abs(liq - 0.19) < 1e-14 and abs(gas - 0.05) < 1e-14
    x = np.arange(nx)
    prof = 0.12 + 0.07 * np.sin(2 * np.pi * x / nx) + 0.01 * np.cos(6 * np.pi * x / nx)
    w = [np.mean([prof[(s + k) % nx] for k in range(20)]) for s in range(nx)]
    liq, gas = R.phase_densities(prof)
    assert abs(liq - max(w)) < 1e-14 and abs(gas - min(w)) < 1e-14
    with pytest.raises(ValueError):
        R.phase_densities(prof, width=0)


class FakeBatch:
    """Per-lattice mean densities and a step clock, for the batched sweeps."""

    def __init__(self, rhos):
        self.rho = list(rhos)
        self.t = 0
        self.log = []

    def step(self, n):
        self.t += n
        self.log.append(("step", n))

    def observables(self, lattice=0):
        return {"rho": self.rho[lattice], "t": self.t}

    def add_density(self, delta, lattice=-1):
        self.rho[lattice] += delta


def test_density_sweeps_follow_each_schedule():
    """An increasing and a decreasing run in one batch, each sampled on its
    own App. C.3 interval (500 steps above rho-bar 0.2, 1500 below)."""
    ts = lambda r: 500 if r > 0.2 + 1e-9 else 1500
    sim = FakeBatch([0.195, 0.21])
    up, down = R.density_sweeps(sim, [dict(lattice=0, rho_start=0.195, rho_end=0.205, delta=0.005, t_sample=ts),
                                      dict(lattice=1, rho_start=0.21, rho_end=0.2, delta=-0.005, t_sample=ts)])
    assert [round(r, 6) for r, _ in up] == [0.195, 0.2, 0.205]
    assert [round(r, 6) for r, _ in down] == [0.21, 0.205, 0.2]
    # each sample taken after its own interval, before its density change
    assert [o["t"] for _, o in up] == [1500, 3000, 3500]
    assert [o["t"] for _, o in down] == [500, 1000, 2500]
    assert all(abs(o["rho"] - r) < 1e-12 for r, o in up + down)
    with pytest.raises(ValueError):
        R.density_sweeps(sim, [dict(lattice=0, rho_start=0.1, rho_end=0.2, delta=-0.01, t_sample=10)])
