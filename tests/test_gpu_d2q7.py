"""D2Q7 (the paper's triangular lattice) on the GPU against the D2Q7 oracle,
element by element on the same seeded inputs, through the C ABI.

Tolerances as for D2Q9 (test_gpu_parity.py): FP32 storage in linearly stable
regimes within 1e-5 over 1000 steps; 16-bit storage within 2e-3 in low-noise
stable regimes; where rounding differences grow (the MIPS spinodal, the CIL
ordered state's direction mode) within 4x the FP32 oracle's own divergence.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from lbmtest import assert_parity, errors, gpu_run, gpu_sim, observables, oracle_run, split_preset, storage_shifts

from test_gpu_parity import _write_state_file

pytestmark = pytest.mark.gpu

SEED = W.seed(7)
Q7 = dict(q=7)
U0_CIL7 = W.PRESETS["CIL_Q7_RHO1"]["B"] - W.PRESETS["CIL_Q7_RHO1"]["A"]
W7 = np.array([0.5] + [1.0 / 12.0] * 6)


@pytest.mark.parametrize("storage", ["f32", "f16s", "bf16s"])
@pytest.mark.parametrize("u_kind", [0, 1, 2])
def test_init_matches_oracle7(storage, u_kind):
    model, d = split_preset("CIL_Q7_RHO1")
    spec = dict(rho_mean=1.0, rho_amp=0.1, u_kind=u_kind, u_amp=0.02, ux0=0.01, uy0=-0.005)
    nx, ny = 72, 40
    sim = gpu_sim(model, d, nx, ny, SEED, spec, storage=storage, lattice_id=17, **Q7)
    got = sim.get_state(host=True).numpy().astype(np.float64)
    sim.close()
    assert got.shape == (7, ny, nx)
    ref = O.init7(nx, ny, SEED, lattice_id=17, **spec, prm=O.params(**d))
    if storage == "f32":
        tol = 2.0 ** -24 * np.abs(ref) * 1.01 + 1e-30
    else:
        rel = 2.0 ** -11 if storage == "f16s" else 2.0 ** -8
        tol = rel * np.abs(ref - storage_shifts(storage, 7)[:, None, None]) * 1.01 + 1e-7
    assert np.all(np.abs(got - ref) <= tol)


STABLE7 = {
    "passive_noise": ("PASSIVE", dict(sigma=0.01), W.INIT_CONFIG1),
    "mips_rho1_stable_C": ("MIPS_Q7_RHO1", dict(C=0.2), W.INIT_CONFIG1),
    "mips_rho1_stable_C_low_noise": ("MIPS_Q7_RHO1", dict(C=0.2, sigma=0.0099), W.INIT_CONFIG1),
    "cil_paper_at_rho1": ("CIL_Q7_PAPER", {}, W.INIT_CONFIG2),
    "mips_paper_at_rho1": ("MIPS_Q7_PAPER", {}, W.INIT_CONFIG2),
    "passive_tau_1p7": ("PASSIVE", dict(tau=1.7, sigma=0.005), W.INIT_CONFIG2),
    "cil_paper_at_rho1_low_noise": ("CIL_Q7_PAPER", dict(sigma=0.0099), W.INIT_CONFIG2),
}


@pytest.mark.parametrize("case", sorted(STABLE7))
def test_step_parity_fp32_1000_steps7(case):
    name, over, spec = STABLE7[case]
    model, d = split_preset(name, **over)
    got = gpu_run(model, d, 64, 64, 1000, SEED, spec, **Q7)
    ref = oracle_run(model, d, 64, 64, 1000, SEED, spec, **Q7)
    e_rho, e_u = errors(got, ref)
    assert e_rho <= 1e-5 and e_u <= 1e-5, (e_rho, e_u)


BF16_MISS7 = pytest.mark.xfail(strict=True, reason="BF16 shifted storage misses the 2e-3 bound here: e_u = "
                                                   "2.31e-3 measured (8 significand bits on noise-sized deviations)")


@pytest.mark.parametrize("storage,case", [("f16s", "mips_rho1_stable_C_low_noise"),
                                          ("f16s", "cil_paper_at_rho1_low_noise"),
                                          ("bf16s", "mips_rho1_stable_C_low_noise"),
                                          pytest.param("bf16s", "cil_paper_at_rho1_low_noise", marks=BF16_MISS7)])
def test_step_parity_16bit_1000_steps7(storage, case):
    """The 2e-3 bound is the one stated for tau = 1 runs with low noise (sigma
    ~ 0.01, as in the D2Q9 test).  The paper's D2Q7 sigma = 1/70 is sqrt 2 above
    the D2Q9 presets', and its MIPS tau = 2 relaxes velocities half as fast;
    both leave BF16 rounding of the shifted populations at about 2e-3, so
    these cases run at tau = 1 and sigma = 0.0099 (the same code path)."""
    name, over, spec = STABLE7[case]
    model, d = split_preset(name, **dict(over, tau=1.0))
    got = gpu_run(model, d, 64, 64, 1000, SEED, spec, storage=storage, **Q7)
    ref = oracle_run(model, d, 64, 64, 1000, SEED, spec, **Q7)
    e_rho, e_u = errors(got, ref)
    assert e_rho <= 2e-3 and e_u <= 2e-3, (e_rho, e_u)


@pytest.mark.parametrize("case", ["mips_rho1", "cil_rho1_ordered", "cil_paper_hysteresis_rho"])
def test_step_parity_fp32_growing_regimes7(case):
    if case == "mips_rho1":
        model, d = split_preset("MIPS_Q7_RHO1")
        spec, steps_list = W.INIT_CONFIG1, (1, 3, 5, 30, 300)
    elif case == "cil_rho1_ordered":
        model, d = split_preset("CIL_Q7_RHO1")
        spec, steps_list = W.init_ordered(U0_CIL7), (100, 1000)
    else:  # the paper's CIL parameters at one of its hysteresis densities
        model, d = split_preset("CIL_Q7_PAPER")
        spec, steps_list = dict(W.INIT_PAPER_CIL, rho_mean=0.2), (100, 500)
    for steps in steps_list:
        got = gpu_run(model, d, 64, 64, steps, SEED, spec, **Q7)
        e, ei = assert_parity(got, model, d, 64, 64, steps, SEED, spec)
        # grid modes grow faster than on D2Q9 (c_s^2 = 1/4 in App. B's rate):
        # the strict bound holds for the first three steps
        if steps <= 3:
            assert max(e) <= 1e-5, (steps, e)


# ------------------------------------------------- ragged sizes and shapes --
SHAPES7 = [(1, 2), (7, 2), (3, 4), (5, 18), (33, 10), (64, 20), (100, 38), (130, 4), (257, 18), (180, 60)]


@pytest.mark.parametrize("nx,ny", SHAPES7)
def test_ragged_sizes_default_shape7(nx, ny):
    cases = (("CIL_Q7_RHO1", {}, 20, W.init_ordered(U0_CIL7)), ("MIPS_Q7_RHO1", {}, 3, W.INIT_CONFIG1),
             ("MIPS_Q7_RHO1", dict(C=0.2), 40, W.INIT_CONFIG1), ("PASSIVE", dict(sigma=0.01), 40, W.INIT_CONFIG2))
    for name, over, steps, spec in cases:
        model, d = split_preset(name, **over)
        got = gpu_run(model, d, nx, ny, steps, SEED, spec, **Q7)
        assert_parity(got, model, d, nx, ny, steps, SEED, spec)


SHAPES_FIXED7 = [(1, 16), (2, 16), (4, 16), (4, 48), (2, 128), (8, 32), (1, 16, 2), (2, 32, 8),
                 (1, 16, 4, 3), (2, 32, 2, 4), (4, 64, 4, 6), (2, 48, 4, 3), (8, 32, 2, 4), (4, 32, 1, 3),
                 (4, 32, 8, 4), (2, 16, 8, 3), (8, 16, 8, 5), (4, 32, 8, 2), (4, 16, 4, 2)]


def staged_refusal7(model, storage, shape):
    """Why lbm_set_tuning refuses a staged D2Q7 shape, or None (as on D2Q9:
    MIPS needs 3 row buffers, 2 with 16-bit storage and its two converted FP32
    rows per warp; the buffers must fit a block's 227 KB)."""
    if len(shape) < 4:
        return None
    vec, _, warps, stages = shape
    eb = 4 if storage == "f32" else 2
    conv = model == "mips" and eb == 2
    if model == "mips" and stages < (2 if conv else 3):
        return "stages"
    smem = stages * (7 * (warps * 32 * vec + 2 * (16 // eb)) * eb + 16) + (2 * 7 * warps * 32 * vec * 4 if conv else 0)
    return "shared memory" if smem > 232448 else None


@pytest.mark.parametrize("shape", SHAPES_FIXED7, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("storage", ["f32", "bf16s"])
@pytest.mark.parametrize("name", ["MIPS_Q7_RHO1", "CIL_Q7_RHO1", "PASSIVE"])
def test_launch_shapes_give_identical_states7(shape, storage, name):
    """Every launch shape -- direct loads (vec, rows, warps) or bulk-copy
    staged rows (vec, rows, warps, stages) -- performs the same per-site
    arithmetic: bitwise equal to the (vec 1, rows 16) shape, and within parity
    of the oracle."""
    if storage == "f32" and shape[0] == 8:
        pytest.skip("vec 8 is a 16-bit storage shape")
    model, d = split_preset(name, **(dict(sigma=0.01) if name == "PASSIVE" else {}))
    nx, ny = 264, 70
    spec = W.INIT_CONFIG1 if model != "cil" else W.init_ordered(U0_CIL7)
    if staged_refusal7(model, storage, shape):
        from paper_1902_00530_gb300 import LBMError
        with pytest.raises(LBMError, match="INVALID_ARG"):
            gpu_run(model, d, nx, ny, 9, SEED, spec, storage=storage, tuning=shape, **Q7)
        return
    base = gpu_run(model, d, nx, ny, 9, SEED, spec, storage=storage, tuning=(1, 16), **Q7)
    got = gpu_run(model, d, nx, ny, 9, SEED, spec, storage=storage, tuning=shape, **Q7)
    np.testing.assert_array_equal(got, base)
    if storage == "f32":
        assert_parity(got, model, d, nx, ny, 9, SEED, spec)


@pytest.mark.parametrize("nx,ny", [(4, 4), (8, 2), (36, 6), (64, 64), (96, 34), (520, 18)])
def test_staged_kernel_small_and_ragged7(nx, ny):
    """Staged D2Q7 shapes on lattices narrower than a strip, with a ragged last
    strip, and with the periodic halo wrapping onto the strip itself."""
    for name, over, steps, spec in (("MIPS_Q7_RHO1", {}, 3, W.INIT_CONFIG1),
                                    ("CIL_Q7_RHO1", {}, 20, W.init_ordered(U0_CIL7))):
        model, d = split_preset(name, **over)
        for shape in ((1, 16, 4, 3), (4, 32, 2, 4), (4, 32, 8, 4)):
            if nx % shape[0]:
                continue
            got = gpu_run(model, d, nx, ny, steps, SEED, spec, tuning=shape, **Q7)
            base = gpu_run(model, d, nx, ny, steps, SEED, spec, tuning=(1, 16), **Q7)
            np.testing.assert_array_equal(got, base)
            assert_parity(got, model, d, nx, ny, steps, SEED, spec)


@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
@pytest.mark.parametrize("nx,ny", [(8, 2), (64, 64), (96, 34), (520, 18)])
def test_staged_mips_16bit_small_and_ragged7(nx, ny, storage):
    """The 16-bit D2Q7 MIPS staged kernel (converted FP32 rows, each staged
    row released a row early) on small and ragged lattices, rings of 2 to 4:
    bitwise the direct kernel's states."""
    model, d = split_preset("MIPS_Q7_RHO1")
    for shape in ((1, 16, 4, 2), (4, 16, 4, 2), (2, 8, 8, 3), (4, 32, 2, 4), (8, 16, 1, 2)):
        if nx % shape[0]:
            continue
        got = gpu_run(model, d, nx, ny, 5, SEED, W.INIT_CONFIG1, storage=storage, tuning=shape, **Q7)
        base = gpu_run(model, d, nx, ny, 5, SEED, W.INIT_CONFIG1, storage=storage, tuning=(1, 16), **Q7)
        np.testing.assert_array_equal(got, base)


@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
def test_sampled_observables_16bit_mips_staged7(storage):
    """Sample steps of the 16-bit D2Q7 MIPS staged kernel (converted rows):
    states bitwise those of the direct kernel, records equal to FP32 rounding
    (each thread's partial sums depend on the launch shape)."""
    model, d = split_preset("MIPS_Q7_RHO1")
    nx, ny, every, steps = 264, 70, 3, 12
    runs = []
    for tuning in ((1, 16), (4, 16, 4, 2), (4, 32, 8, 2)):
        sim = gpu_sim(model, d, nx, ny, SEED, W.INIT_CONFIG1, storage=storage, sample_every=every, ring=16,
                      tuning=tuning, **Q7)
        sim.step(steps)
        runs.append((sim.observable_series(), sim.get_state(host=True).numpy()))
        sim.close()
    (s0, f0) = runs[0]
    assert [r["t"] for r in s0] == list(range(every, steps + 1, every))
    for series, f in runs[1:]:
        np.testing.assert_array_equal(f, f0)
        for a, b in zip(series, s0):
            for key in ("mass", "phi", "drho_y", "drho_x", "var_rho", "zeta"):
                assert a[key] == pytest.approx(b[key], rel=1e-6, abs=1e-6), (key, a[key], b[key])


# ---------------------------------------------------------- noise stream ---
@pytest.mark.parametrize("t,lattice_id,seed", [(0, 0, SEED), (7, 3, 12345), (2 ** 31 + 12345, 2 ** 24 - 1,
                                                                                  2 ** 63 + 99)])
def test_noise_stream_matches_oracle7(tmp_path, t, lattice_id, seed):
    """From a uniform rest state one step adds exactly the zero-sum noise
    sigma (s_i - mean s) of the oracle's 16-bit variates."""
    from paper_1902_00530_gb300 import Lattice, Simulation
    nx, ny, rho, sigma = 40, 24, 40.0, 0.5
    f0 = np.broadcast_to((W7 * rho)[:, None, None], (7, ny, nx)).astype(np.float32)
    path = tmp_path / "rest7.lbm"
    _write_state_file(path, f0, t, seed, lattice_id, 0)
    sim = Simulation([Lattice(nx, ny, "f32", lattice_id, "d2q7")], ["passive"], [dict(tau=1.3, sigma=sigma)])
    sim.load(str(path))
    assert sim.time == t
    sim.step(1)
    got = sim.get_state(host=True).numpy().astype(np.float64) - (W7 * rho)[:, None, None]
    sim.close()
    for (x, y) in [(0, 0), (1, 0), (nx - 1, ny - 1), (17, 5), (3, 20)]:
        s = O.noise_variates7(seed, x, y, t, lattice_id)
        np.testing.assert_allclose(got[:, y, x], sigma * (s - s.mean()), rtol=0, atol=1e-5)


# ------------------------------------------------------------ observables --
def test_sampled_observables_match_oracle7():
    model, d = split_preset("CIL_Q7_RHO1")
    nx, ny, every, steps = 96, 40, 10, 60
    spec = W.init_ordered(U0_CIL7, rho_amp=0.05, u_amp=0.02)
    sim = gpu_sim(model, d, nx, ny, SEED, spec, sample_every=every, ring=16, **Q7)
    sim.step(steps)
    series = sim.observable_series()
    now = sim.observables()
    sim.close()
    assert [r["t"] for r in series] == list(range(every, steps + 1, every))
    p = O.params(**d)
    f = O.init7(nx, ny, SEED, **spec, prm=p)
    for k, rec in enumerate(series):
        f = O.run7(f, model, p, SEED, k * every, every)
        ref = O.observables7(f, B=d["B"])
        assert abs(rec["mass"] - ref["mass"]) / ref["mass"] < 1e-6
        for key in ("phi", "drho_y", "drho_x", "zeta"):
            assert abs(rec[key] - ref[key]) < 2e-6, (key, rec[key], ref[key])
        assert abs(rec["var_rho"] - ref["var_rho"]) < 1e-7
    for key in ("mass", "phi", "drho_y", "drho_x", "var_rho", "zeta"):
        assert now[key] == pytest.approx(series[-1][key], rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
def test_observables_16bit_storage7(storage):
    model, d = split_preset("MIPS_Q7_PAPER")
    sim = gpu_sim(model, d, 128, 64, SEED, W.INIT_CONFIG2, storage=storage, **Q7)
    sim.step(50)
    ob = sim.observables()
    f = sim.get_state(host=True).numpy().astype(np.float64)
    sim.close()
    own = observables(f)
    assert abs(ob["mass"] - own["mass"]) / own["mass"] < 1e-7
    assert abs(ob["drho_y"] - own["drho_y"]) < 1e-6 and abs(ob["var_rho"] - own["var_rho"]) < 1e-7


def test_moments_match_oracle7():
    model, d = split_preset("MIPS_Q7_RHO1", C=0.2)
    nx, ny = 80, 48
    sim = gpu_sim(model, d, nx, ny, SEED, W.INIT_CONFIG1, **Q7)
    sim.step(25)
    rho, ux, uy = (a.cpu().numpy().astype(np.float64) for a in sim.moments())
    sim.close()
    rr, uxr, uyr = O.moments7(oracle_run(model, d, nx, ny, 25, SEED, W.INIT_CONFIG1, **Q7))
    assert np.abs(rho - rr).max() < 1e-5
    assert max(np.abs(ux - uxr).max(), np.abs(uy - uyr).max()) < 1e-5


@pytest.mark.parametrize("name,over,spec", [("PASSIVE", dict(sigma=0.0099), W.INIT_CONFIG2),
                                             ("MIPS_Q7_PAPER", {}, W.INIT_CONFIG2),
                                             ("MIPS_Q7_RHO1", {}, W.INIT_CONFIG1)])
def test_mass_conservation_fp32_7(name, over, spec):
    """Mass over 1000 steps within 1e-6 or the FP32 oracle's own drift."""
    model, d = split_preset(name, **over)
    nx, ny = 128, 64
    sim = gpu_sim(model, d, nx, ny, SEED, spec, **Q7)
    m0 = sim.observables()["mass"]
    sim.step(1000)
    m1 = sim.observables()["mass"]
    sim.close()
    p = O.params(**d)
    f = O.init7(nx, ny, SEED, **spec, prm=p, bits=32)
    g = O.run7(f, model, p, SEED, 0, 1000, bits=32)
    drift32 = abs(O.observables7(g.astype(np.float64))["mass"] - O.observables7(f.astype(np.float64))["mass"])
    assert abs(m1 - m0) <= max(1e-6 * m0, 4 * drift32), (m1 - m0, drift32)


# ---------------------------------------------------- symmetry and batches --
@pytest.mark.parametrize("name", ["MIPS_Q7_RHO1", "CIL_Q7_RHO1"])
def test_density_rescaling_bitwise_gpu7(name):
    model, d = split_preset(name)
    d2 = dict(d, C=d["C"] / 2, rho_star=d["rho_star"] * 2, A=d["A"] / 4, sigma=d["sigma"] * 2)
    spec = dict(W.INIT_CONFIG2)
    spec2 = dict(spec, rho_mean=2 * spec["rho_mean"])
    a = gpu_run(model, d, 96, 48, 200, SEED, spec, **Q7)
    b = gpu_run(model, d2, 96, 48, 200, SEED, spec2, **Q7)
    np.testing.assert_array_equal(b, 2 * a)


def test_mixed_batch_equals_solo_runs7():
    """D2Q7 and D2Q9 lattices in one batch (separate launch groups) evolve as
    they do alone."""
    from paper_1902_00530_gb300 import Lattice, Simulation
    cfg = [(Lattice(64, 64, "f32", 0, "d2q7"), "cil", split_preset("CIL_Q7_RHO1")[1], W.INIT_CONFIG2),
           (Lattice(96, 32, "f32", 1), "mips", split_preset("MIPS_RHO1")[1], W.INIT_CONFIG1),
           (Lattice(90, 30, "f32", 2, "d2q7"), "mips", split_preset("MIPS_Q7_RHO1")[1], W.INIT_CONFIG1),
           (Lattice(128, 40, "bf16s", 3, "d2q7"), "cil", split_preset("CIL_Q7_RHO1")[1], W.INIT_PAPER_CIL)]
    sim = Simulation([c[0] for c in cfg], [c[1] for c in cfg], [c[2] for c in cfg])
    sim.init(SEED, [c[3] for c in cfg])
    sim.step(60)
    batch = [sim.get_state(k, host=True).numpy() for k in range(len(cfg))]
    sim.close()
    for k, (lat, model, d, spec) in enumerate(cfg):
        solo = gpu_run(model, d, lat.nx, lat.ny, 60, SEED, spec, storage=lat.storage, lattice_id=lat.id,
                       q=lat.q)
        np.testing.assert_array_equal(batch[k], solo.astype(np.float32))


def test_resume_is_bit_exact7(tmp_path):
    model, d = split_preset("MIPS_Q7_RHO1")
    sim = gpu_sim(model, d, 64, 48, SEED, W.INIT_CONFIG1, **Q7)
    sim.step(30)
    sim.save(str(tmp_path / "s7.lbm"))
    sim.step(30)
    full = sim.get_state(host=True).numpy()
    sim.close()
    sim = gpu_sim(model, d, 64, 48, SEED + 1, W.INIT_CONFIG2, **Q7)
    sim.load(str(tmp_path / "s7.lbm"))
    assert sim.time == 30
    sim.step(30)
    np.testing.assert_array_equal(sim.get_state(host=True).numpy(), full)
    sim.close()


def test_graphs_on_off_identical7():
    model, d = split_preset("MIPS_Q7_RHO1")
    a = gpu_run(model, d, 64, 64, 77, SEED, W.INIT_CONFIG2, graphs=True, sample_every=10, ring=8, **Q7)
    b = gpu_run(model, d, 64, 64, 77, SEED, W.INIT_CONFIG2, graphs=False, sample_every=10, ring=8, **Q7)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_add_density_matches_oracle7(storage):
    """App. C.2 as printed for D2Q7: delta rho-bar / 7 added to every f_i."""
    model, d = split_preset("CIL_Q7_PAPER")
    nx, ny, spec = 64, 48, W.INIT_CONFIG2
    sim = gpu_sim(model, d, nx, ny, SEED, spec, storage=storage, **Q7)
    sim.step(20)
    m0 = sim.observables()["mass"]
    sim.add_density(0.05)
    assert abs(sim.observables()["mass"] - (m0 + 0.05 * nx * ny)) / m0 < 1e-6
    sim.step(20)
    got = sim.get_state(host=True).numpy().astype(np.float64)
    sim.close()
    p = O.params(**d)
    f = O.run7(O.init7(nx, ny, SEED, **spec, prm=p), model, p, SEED, 0, 20)
    f = O.run7(O.add_density7(f, 0.05), model, p, SEED, 20, 20)
    assert max(errors(got, f)) <= (1e-5 if storage == "f32" else 2e-3)


def test_set_state_round_trip7():
    model, d = split_preset("PASSIVE", sigma=0.01)
    f = O.init7(40, 20, SEED, **W.INIT_CONFIG2, prm=O.params(**d)).astype(np.float32)
    from paper_1902_00530_gb300 import Lattice, Simulation
    for storage in ("f32", "bf16s"):
        sim = Simulation([Lattice(40, 20, storage, 0, "d2q7")], [model], [d])
        sim.set_state(f)
        g = sim.get_state(host=True).numpy()
        sim.close()
        if storage == "f32":
            np.testing.assert_array_equal(g, f)
        else:
            assert np.abs(g - f).max() <= 2.0 ** -8 * np.abs(f - storage_shifts(storage, 7)[:, None, None]).max() * 1.01 + 1e-7


# ---------------------------------------------- full size, sampled sites ---
@pytest.mark.parametrize("storage,preset", [("f32", "MIPS_Q7_RHO1"), ("bf16s", "MIPS_Q7_PAPER")])
def test_full_size_sampled_parity7(storage, preset):
    """8192^2 D2Q7 in the tuned launch shape: sampled sites against oracle
    windows at the same global coordinates (even y offsets keep the row
    parity), exact inside the light cone.  16-bit storage is checked at
    tau = 1, where the stated 2e-3 bound applies (see the 16-bit test)."""
    from paper_1902_00530_gb300 import Lattice, Simulation
    model, d = split_preset(preset, **({} if storage == "f32" else dict(tau=1.0)))
    N, k, R = 8192, 3, 10
    sim = Simulation([Lattice(N, N, storage, 0, "d2q7")], [model], [d])
    sim.init(SEED, [W.INIT_CONFIG1])
    sim.tune()
    sim.step(k)
    rho, ux, uy = (a.cpu().numpy().astype(np.float64) for a in sim.moments())
    sim.close()
    tol = 1e-5 if storage == "f32" else 2e-3
    p = O.params(**d)
    for (cx, cy) in [(0, 0), (N - 1, N - 2), (0, N // 2), (4097, 4), (1234, 5678), (N - 3, 18)]:
        w = 2 * R + 2
        win = (cx - R, cy - R, N, N)  # cy - R even
        f = O.run7(O.init7(w, w, SEED, **W.INIT_CONFIG1, prm=p, window=win), model, p, SEED, 0, k, window=win)
        rr, uxr, uyr = O.moments7(f)
        m = R - 2 * k - 1
        ys = [(cy + j) % N for j in range(-m, m + 1)]
        xs = [(cx + i) % N for i in range(-m, m + 1)]
        sl = slice(R - m, R + m + 1)
        assert np.abs(rho[np.ix_(ys, xs)] - rr[sl, sl]).max() / rr.mean() <= tol
        du = max(np.abs(ux[np.ix_(ys, xs)] - uxr[sl, sl]).max(), np.abs(uy[np.ix_(ys, xs)] - uyr[sl, sl]).max())
        assert du / max(np.hypot(uxr, uyr).max(), 1e-3) <= tol
