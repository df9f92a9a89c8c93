"""Seeded synthetic workloads: parameter presets, initial-state recipes, seeds.

This module holds inputs only -- numbers and recipes, none of the method's
arithmetic.  The tests, the oracle leg and ``bench.py`` take their inputs from
here; neither the oracle nor the CUDA path imports the other.

Presets.  The paper's parameters (Table "ParametersMIPS", App. C.1; App. C.2)
live at mean densities 0.1-0.35.  The configurations here run at mean density
about 1, so each paper preset appears twice:

* ``*_PAPER_LITERAL``: the paper's numbers as printed.  At rho ~ 1 they are
  degenerate (MIPS: rho > rho* so u* = 0; CIL: B < A rho^2 so U0 = 0).
* ``*_RHO1``: the same physics moved to rho ~ 1 by the model's exact
  density-rescaling symmetry (f, rho, C, rho*, A, sigma) -> (s f, s rho, C/s,
  s rho*, A/s^2, s sigma) with s = 1/(the paper's mean density).

Noise amplitude on D2Q9.  The paper's noise gives <h_x^2> = c^2 sigma^2 on D2Q7
(Sec. 7); with the same uniform eta~ on D2Q9 the momentum noise is 2 sigma^2,
so a paper sigma is carried over as sigma / sqrt(2).

D2Q7 presets (``*_Q7_*``) are for the paper's own triangular lattice, where
its numbers apply unchanged: ``*_Q7_PAPER`` as printed (run at the paper's
mean densities) and ``*_Q7_RHO1`` rescaled to rho ~ 1 as above.
"""
from __future__ import annotations

import math

SEED_BASE = 190200530


def seed(k: int) -> int:
    """Seed of configuration k (1-based)."""
    return SEED_BASE + k


SQRT2 = math.sqrt(2.0)

# paper values (Table ParametersMIPS; stills (b)-(d) sigma = 0.014; App. C.1 rho-bar = 0.12)
_MIPS_C, _MIPS_RHO_STAR, _MIPS_UMAX, _MIPS_SIGMA, _MIPS_RHOBAR = 50.0, 0.2, 0.3, 0.014, 0.12
_MIPS_TAU = 2.0  # Table ParametersMIPS; the D2Q9 presets use tau = 1
# paper values (App. C.2: B = 0.3, tau = 1, sigma = 1/70; Fig. Hysteresis A = 2; HO snapshot rho-bar 0.185)
_CIL_A, _CIL_B, _CIL_SIGMA, _CIL_RHOBAR = 2.0, 0.3, 1.0 / 70.0, 0.185

PRESETS = {
    "MIPS_PAPER_LITERAL": dict(model="mips", tau=1.0, sigma=_MIPS_SIGMA / SQRT2, C=_MIPS_C,
                               rho_star=_MIPS_RHO_STAR, u_max=_MIPS_UMAX, A=0.0, B=0.0),
    "MIPS_RHO1": dict(model="mips", tau=1.0, sigma=_MIPS_SIGMA / _MIPS_RHOBAR / SQRT2,
                      C=_MIPS_C * _MIPS_RHOBAR, rho_star=_MIPS_RHO_STAR / _MIPS_RHOBAR,
                      u_max=_MIPS_UMAX, A=0.0, B=0.0),
    "CIL_PAPER_LITERAL": dict(model="cil", tau=1.0, sigma=_CIL_SIGMA / SQRT2, C=0.0, rho_star=1.0,
                              u_max=1.0, A=_CIL_A, B=_CIL_B),
    "CIL_RHO1": dict(model="cil", tau=1.0, sigma=_CIL_SIGMA / _CIL_RHOBAR / SQRT2, C=0.0,
                     rho_star=1.0, u_max=1.0, A=_CIL_A * _CIL_RHOBAR ** 2, B=_CIL_B),
    "PASSIVE": dict(model="passive", tau=1.0, sigma=0.0, C=0.0, rho_star=1.0, u_max=1.0,
                    A=0.0, B=0.0),
    # D2Q7: the paper's lattice, its parameters as printed (MIPS: Table ParametersMIPS, tau = 2)
    "MIPS_Q7_PAPER": dict(model="mips", tau=_MIPS_TAU, sigma=_MIPS_SIGMA, C=_MIPS_C, rho_star=_MIPS_RHO_STAR,
                          u_max=_MIPS_UMAX, A=0.0, B=0.0),
    "MIPS_Q7_RHO1": dict(model="mips", tau=_MIPS_TAU, sigma=_MIPS_SIGMA / _MIPS_RHOBAR, C=_MIPS_C * _MIPS_RHOBAR,
                         rho_star=_MIPS_RHO_STAR / _MIPS_RHOBAR, u_max=_MIPS_UMAX, A=0.0, B=0.0),
    "CIL_Q7_PAPER": dict(model="cil", tau=1.0, sigma=_CIL_SIGMA, C=0.0, rho_star=1.0, u_max=1.0,
                         A=_CIL_A, B=_CIL_B),
    "CIL_Q7_RHO1": dict(model="cil", tau=1.0, sigma=_CIL_SIGMA / _CIL_RHOBAR, C=0.0, rho_star=1.0,
                        u_max=1.0, A=_CIL_A * _CIL_RHOBAR ** 2, B=_CIL_B),
}

# the paper's mean densities for its D2Q7 runs (App. C.1 MIPS phase diagram;
# App. C.2 CIL homogeneous-ordered snapshot) and boxes (App. C)
MIPS_RHOBAR_PAPER, CIL_RHOBAR_PAPER = _MIPS_RHOBAR, _CIL_RHOBAR
BOX_CIL_PAPER = (180, 60)
BOX_MIPS_PHASE_PAPER = (90, 30)


def preset(name: str, **overrides) -> dict:
    d = dict(PRESETS[name])
    d.update(overrides)
    return d


# Initial-state recipes (App. C.2 style): rho = rho_mean (1 + rho_amp (2U - 1));
# u_kind 0: (ux0, uy0) + u_amp (2U - 1) per component; 1: (ux0, uy0) + u_amp * random
# unit vector; 2: U0(rho) * random unit vector (the paper's CIL initialisation).
INIT_CONFIG1 = dict(rho_mean=1.0, rho_amp=0.01, u_kind=0, u_amp=1e-3, ux0=0.0, uy0=0.0)
INIT_CONFIG2 = dict(rho_mean=1.0, rho_amp=0.1, u_kind=1, u_amp=0.01, ux0=0.0, uy0=0.0)
INIT_PAPER_CIL = dict(rho_mean=1.0, rho_amp=0.1, u_kind=2, u_amp=0.0, ux0=0.0, uy0=0.0)


def init_ordered(u0: float, rho_amp: float = 0.01, u_amp: float = 1e-3) -> dict:
    """Homogeneous ordered state along x with small seeded perturbations."""
    return dict(rho_mean=1.0, rho_amp=rho_amp, u_kind=0, u_amp=u_amp, ux0=u0, uy0=0.0)


# Configurations (lattice sizes, step counts) of the workloads.
CONFIG1 = dict(nx=64, ny=64, steps=1000, init=INIT_CONFIG1)              # parity, MIPS
CONFIG2 = dict(nx=1024, ny=1024, steps=10_000, sample_every=100, init=INIT_CONFIG2,
               preset="CIL_RHO1")                                         # CIL + observables
CONFIG3 = dict(nx=8192, ny=8192, steps=1000, crop=512, init=INIT_CONFIG1,
               preset="MIPS_RHO1")                                        # precision / throughput
CONFIG4 = dict(n=256, side=256, steps=20_000, rho_means=[0.5 + i / 15.0 for i in range(16)],
               activities=[0.1 * i / 15.0 for i in range(16)], preset="CIL_RHO1",
               init=INIT_CONFIG2)                                         # uniform batch
CONFIG5 = dict(n=64, sides=(128, 256, 512, 1024, 2048), steps=20_000, sample_every=100)


def ragged_batch(seed_value: int | None = None):
    """Side lengths and models of the ragged batch, drawn from a seed."""
    import numpy as np
    rng = np.random.default_rng(seed(5) if seed_value is None else seed_value)
    sides = rng.choice(CONFIG5["sides"], size=CONFIG5["n"])
    models = rng.integers(0, 2, size=CONFIG5["n"])
    return [(int(s), "MIPS_RHO1" if m == 0 else "CIL_RHO1") for s, m in zip(sides, models)]
