"""Persistent launches (lbm_set_persistent) against one launch per step.

A persistent launch runs many steps of a launch group in one kernel, each step
the same direct-kernel update of App. A.2, so every state, sampled observable
series and on-demand record must be bitwise those of the per-step launches:
across the three closures, the noise forms (none, all, mixed within a group),
storage types, both lattices (D2Q9 and the paper's D2Q7), launch shapes
(blocks spanning strip rows, lattices of one or two strip rows, a staged shape
the persistent launch leaves alone), lattice groups smaller and larger than
the batch, sample steps at every phase of a persistent stretch, with and
without CUDA graphs.
"""
import numpy as np
import pytest

import workloads as W
from lbmtest import split_preset

pytestmark = pytest.mark.gpu
SEED = W.seed(11)

# (nx, ny, preset, overrides, init): three launch groups per storage type --
# CIL with noise in some lattices only, MIPS with noise, passive without
MIXED = [(64, 64, "CIL_RHO1", {}, W.INIT_CONFIG2),
         (96, 40, "MIPS_RHO1", {}, W.INIT_CONFIG1),
         (136, 24, "CIL_RHO1", dict(B=0.05, sigma=0.0), dict(W.INIT_CONFIG2, rho_mean=0.7)),
         (40, 72, "MIPS_RHO1", {}, W.INIT_CONFIG1),
         (72, 56, "PASSIVE", {}, W.INIT_CONFIG2),
         (256, 32, "CIL_RHO1", {}, W.INIT_CONFIG2),
         (64, 16, "PASSIVE", {}, W.INIT_CONFIG1)]


# the paper's D2Q7 lattice (ny even), with one D2Q9 lattice in the same batch
MIXED7 = [(64, 32, "CIL_Q7_RHO1", {}, W.INIT_CONFIG2, "d2q7"),
          (96, 40, "MIPS_Q7_RHO1", dict(C=0.2), W.INIT_CONFIG1, "d2q7"),
          (136, 24, "CIL_Q7_RHO1", dict(B=0.05, sigma=0.0), dict(W.INIT_CONFIG2, rho_mean=0.7), "d2q7"),
          (72, 56, "PASSIVE", dict(sigma=0.01), W.INIT_CONFIG2, "d2q7"),
          (180, 60, "CIL_Q7_PAPER", {}, dict(W.INIT_PAPER_CIL, rho_mean=0.185), "d2q7"),
          (64, 48, "CIL_RHO1", {}, W.INIT_CONFIG2, "d2q9")]


def _run(storage, persistent, tuning, l2_mib=1, graphs=True, every=9, calls=(37, 28), cfg=MIXED):
    from paper_1902_00530_gb300 import Lattice, Simulation
    lats, mods, prms, specs = [], [], [], []
    for k, (nx, ny, name, over, init, *vs) in enumerate(cfg):
        model, d = split_preset(name, **over)
        lats.append(Lattice(nx, ny, storage, k, vs[0] if vs else "d2q9"))
        mods.append(model)
        prms.append(d)
        specs.append(init)
    sim = Simulation(lats, mods, prms, sample_every=every, ring_capacity=64 if every else 0)
    sim.set_tuning(1, *tuning)
    sim.set_graphs(graphs)
    sim.set_persistent(persistent, l2_mib)
    sim.init(SEED, specs)
    launches = []
    for n in calls:
        sim.step(n)
        launches.append(sim.last_launch_count())
    out = dict(states=[sim.get_state(k, host=True).numpy() for k in range(len(cfg))],
               obs=[sim.observables(k) for k in range(len(cfg))], launches=launches)
    if every:
        out["series"] = [sim.observable_series(k) for k in range(len(cfg))]
    sim.close()
    return out


def _assert_same(a, b):
    for k, (x, y) in enumerate(zip(a["states"], b["states"])):
        np.testing.assert_array_equal(x, y, err_msg=f"lattice {k}")
    assert a["obs"] == b["obs"]
    assert a.get("series") == b.get("series")


SHAPES = [(1, 8, 4, 0), (4, 8, 4, 0), (2, 16, 8, 0), (1, 32, 1, 0), (4, 16, 4, 3)]


@pytest.mark.parametrize("tuning", SHAPES)
@pytest.mark.parametrize("storage", ["f32", "f16s", "bf16s"])
def test_persistent_equals_per_step_launches(storage, tuning):
    ref = _run(storage, False, tuning)
    got = _run(storage, True, tuning)
    _assert_same(got, ref)
    if tuning[3] == 0:  # direct groups: a stretch of plain steps is one launch
        assert sum(got["launches"]) < sum(ref["launches"])
    else:               # staged groups are left to the per-step launches
        assert got["launches"] == ref["launches"]


@pytest.mark.parametrize("tuning", [(1, 8, 4, 0), (4, 8, 4, 0), (2, 16, 8, 0), (1, 32, 1, 0)])
@pytest.mark.parametrize("storage", ["f32", "bf16s"])
def test_persistent_d2q7_equals_per_step_launches(storage, tuning):
    """The paper's D2Q7 lattice: its direct kernel's strip update in the
    persistent launch, beside a D2Q9 group of the same batch."""
    ref = _run(storage, False, tuning, cfg=MIXED7)
    got = _run(storage, True, tuning, cfg=MIXED7)
    _assert_same(got, ref)
    assert sum(got["launches"]) < sum(ref["launches"])


@pytest.mark.parametrize("graphs", [True, False])
@pytest.mark.parametrize("l2_mib", [0, 1, 3])
def test_persistent_lattice_groups_and_graphs(graphs, l2_mib):
    tuning = (2, 8, 4, 0)
    ref = _run("f32", False, tuning, graphs=True)
    got = _run("f32", True, tuning, l2_mib=l2_mib, graphs=graphs)
    _assert_same(got, ref)


@pytest.mark.parametrize("every", [0, 1, 2, 5])
def test_persistent_sampling_phases(every):
    tuning = (1, 8, 4, 0)
    calls = (3, 1, 2, 41, 17)
    ref = _run("f16s", False, tuning, every=every, calls=calls)
    got = _run("f16s", True, tuning, every=every, calls=calls)
    _assert_same(got, ref)


def test_persistent_launch_count_and_profile():
    from paper_1902_00530_gb300 import Lattice, Simulation
    model, d = split_preset("CIL_RHO1")
    sim = Simulation([Lattice(128, 64, "f32", 0), Lattice(64, 64, "f32", 1)], [model] * 2, [d] * 2)
    sim.set_tuning(1, 4, 8, 4, 0)
    sim.set_persistent(True)
    sim.init(SEED, [W.INIT_CONFIG2] * 2)
    sim.step(50)
    assert sim.last_launch_count() == 2        # one persistent launch and the time advance
    sim.set_profiling(True)
    sim.step(20)
    prof = sim.profile_read()
    assert prof["step_launches"] == 20         # a persistent launch counts the steps it runs
    assert prof["step_ms"] > 0.0
    sim.set_profiling(False)
    sim.close()


def _config4_sim(storage, persistent):
    from paper_1902_00530_gb300 import Lattice, Simulation
    c4 = W.CONFIG4
    d = W.preset(c4["preset"])
    model = d.pop("model")
    lats, prms, specs = [], [], []
    for i, rm in enumerate(c4["rho_means"]):
        for j, act in enumerate(c4["activities"]):
            lats.append(Lattice(c4["side"], c4["side"], storage, i * 16 + j))
            prms.append(dict(d, B=act))
            specs.append(dict(c4["init"], rho_mean=rm))
    sim = Simulation(lats, [model] * len(lats), prms, sample_every=25, ring_capacity=8)
    sim.set_tuning(1, 4, 8, 4, 0)
    sim.set_persistent(persistent)
    sim.init(W.seed(4), specs)
    return sim


@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_persistent_uniform_batch_256_lattices(storage):
    """The 256-lattice 256^2 CIL batch on a density x activity grid: every
    lattice and its observable series bitwise as with per-step launches."""
    import torch
    a = _config4_sim(storage, True)
    b = _config4_sim(storage, False)
    for s in (a, b):
        s.step(60)
    for k in range(256):
        assert torch.equal(a.get_state(k), b.get_state(k)), k
        assert a.observable_series(k) == b.observable_series(k), k
    a.close()
    b.close()


# a CIL group of 2^20 sites (the least the tuner considers for persistent
# launches) beside the small MIPS and passive groups of MIXED
AUTO = [(256, 256, "CIL_RHO1", dict(B=0.05 + 0.02 * k), dict(W.INIT_CONFIG2, rho_mean=0.8 + 0.03 * k))
        for k in range(16)] + [c for c in MIXED if c[2] != "CIL_RHO1"]


@pytest.mark.parametrize("storage", ["f32", "bf16s"])
def test_persistent_auto_chosen_by_the_tuner(storage):
    """Mode 2: the tuner times each direct shape per step and persistent (the
    persistent timing form recomputes the current step into the spare buffer)
    and keeps the faster; whatever it keeps, the states equal the per-step
    run's, so the tuning itself left the state untouched.  The two runs' tuners
    may keep different launch shapes, and the FP64 observable sums are
    grouped by the shape, so across shapes the series agree to FP64 rounding
    (amplified in the variance and the polar order, differences of nearly
    equal sums), zeta to the FP32 rounding of a lane's sum of |j|."""
    from paper_1902_00530_gb300 import Lattice, Simulation

    def run(mode):
        lats, mods, prms, specs = [], [], [], []
        for k, (nx, ny, name, over, init) in enumerate(AUTO):
            model, d = split_preset(name, **over)
            lats.append(Lattice(nx, ny, storage, k))
            mods.append(model)
            prms.append(d)
            specs.append(init)
        sim = Simulation(lats, mods, prms, sample_every=9, ring_capacity=16)
        sim.set_persistent(mode)
        sim.init(SEED, specs)
        sim.step(37)
        sim.step(28)
        out = [sim.get_state(k, host=True).numpy() for k in range(len(AUTO))]
        series = [sim.observable_series(k) for k in range(len(AUTO))]
        forms = [sim.get_persistent(k) for k in range(len(AUTO))]
        sim.close()
        return out, series, forms

    a, sa, fa = run("auto")
    b, sb, fb = run(0)
    assert not any(fb)
    assert not any(fa[16:])  # groups under 2^20 sites stay on one launch per step
    for k in range(len(AUTO)):
        np.testing.assert_array_equal(a[k], b[k], err_msg=f"lattice {k}")
        assert len(sa[k]) == len(sb[k])
        for ra, rb in zip(sa[k], sb[k]):
            assert ra["t"] == rb["t"]
            for key in ("mass", "phi", "drho_y", "drho_x", "var_rho"):
                assert ra[key] == pytest.approx(rb[key], rel=1e-9, abs=1e-15), (k, ra["t"], key)
            # zeta's sum of |j| (magnitudes, no cancellation) is a lane's FP32 sum of its sites
            assert ra["zeta"] == pytest.approx(rb["zeta"], rel=1e-6, abs=1e-12), (k, ra["t"], "zeta")
