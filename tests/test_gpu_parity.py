"""GPU path vs the FP64 oracle, element by element on the same seeded inputs.

Tolerances (relative errors e_rho, e_u as defined in lbmtest.errors):
  FP32 storage, linearly stable regimes, 1000 steps   <= 1e-5
  FP16/BF16 shifted storage, stable regimes            <= 2e-3
  regimes where rounding differences grow -- the MIPS spinodal (growth about
  0.6 per step at the rescaled preset), the CIL ordered state (marginal
  direction mode), the passive model (conserved momentum): within 4x the
  oracle's own FP32-vs-FP64 divergence at the same step; for 16-bit storage,
  steady-state observables within 1 % or 3 standard errors.
"""
import math
import struct

import numpy as np
import pytest

import oracle as O
import workloads as W
from lbmtest import assert_parity, errors, gpu_run, gpu_sim, oracle_run, split_preset, storage_shifts

pytestmark = pytest.mark.gpu

SEED = W.seed(1)
U0_CIL = W.PRESETS["CIL_RHO1"]["B"] - W.PRESETS["CIL_RHO1"]["A"]  # U0 at rho = 1


# ------------------------------------------------------------------ init ----
@pytest.mark.parametrize("storage", ["f32", "f16s", "bf16s"])
@pytest.mark.parametrize("u_kind", [0, 1, 2])
def test_init_matches_oracle(storage, u_kind):
    """App. C.2 initial state: FP64 f^SS rounded once to the storage type."""
    model, d = split_preset("CIL_RHO1")
    spec = dict(rho_mean=1.0, rho_amp=0.1, u_kind=u_kind, u_amp=0.02, ux0=0.01, uy0=-0.005)
    nx, ny = 72, 40
    sim = gpu_sim(model, d, nx, ny, SEED, spec, storage=storage, lattice_id=17)
    got = sim.get_state(host=True).numpy().astype(np.float64)
    sim.close()
    ref = O.init(nx, ny, SEED, lattice_id=17, **spec, prm=O.params(**d))
    if storage == "f32":
        tol = 2.0 ** -24 * np.abs(ref) * 1.01 + 1e-30
    else:
        shift = storage_shifts(storage)[:, None, None]
        rel = 2.0 ** -11 if storage == "f16s" else 2.0 ** -8
        tol = rel * np.abs(ref - shift) * 1.01 + 1e-7
    assert np.all(np.abs(got - ref) <= tol)


# ------------------------------------------------------ stable-regime parity
STABLE = {
    # name: (preset, overrides, init spec)
    "passive_noise": ("PASSIVE", dict(sigma=0.01), W.INIT_CONFIG1),
    "mips_paper_literal": ("MIPS_PAPER_LITERAL", {}, W.INIT_CONFIG1),
    "mips_rho1_stable_C": ("MIPS_RHO1", dict(C=0.2), W.INIT_CONFIG1),
    "cil_paper_literal": ("CIL_PAPER_LITERAL", {}, W.INIT_CONFIG2),
    "passive_tau_1p7": ("PASSIVE", dict(tau=1.7, sigma=0.005), W.INIT_CONFIG2),
    # tau > 2: 1/tau below 1/2, rounded by the host so that 1 - 1/tau is exact
    "passive_tau_3": ("PASSIVE", dict(tau=3.0, sigma=0.005), W.INIT_CONFIG2),
    "mips_rho1_stable_C_low_noise": ("MIPS_RHO1", dict(C=0.2, sigma=0.0099), W.INIT_CONFIG1),
}
GROWING = {
    "cil_rho1_ordered": ("CIL_RHO1", {}, W.init_ordered(U0_CIL)),
    "mips_rho1": ("MIPS_RHO1", {}, W.INIT_CONFIG1),
}


@pytest.mark.parametrize("case", sorted(STABLE))
def test_step_parity_fp32_1000_steps(case):
    name, over, spec = STABLE[case]
    model, d = split_preset(name, **over)
    got = gpu_run(model, d, 64, 64, 1000, SEED, spec)
    ref = oracle_run(model, d, 64, 64, 1000, SEED, spec)
    e_rho, e_u = errors(got, ref)
    assert e_rho <= 1e-5 and e_u <= 1e-5, (e_rho, e_u)


@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
@pytest.mark.parametrize("case", ["mips_paper_literal", "cil_paper_literal", "mips_rho1_stable_C_low_noise"])
def test_step_parity_16bit_1000_steps(storage, case):
    """Low-noise, linearly stable regimes (sigma ~ 0.01).  At the rescaled
    presets' noise (sigma ~ 0.05-0.08) the shifted populations carry
    deviations of the order of sigma, the 16-bit store rounds them to 2^-11
    (FP16) or 2^-8 (BF16) of that, and the error is measured on steady-state
    observables instead (test_16bit_steady_state_observables); so is the
    passive model, whose conserved momentum accumulates rounding."""
    name, over, spec = STABLE[case]
    model, d = split_preset(name, **over)
    got = gpu_run(model, d, 64, 64, 1000, SEED, spec, storage=storage)
    ref = oracle_run(model, d, 64, 64, 1000, SEED, spec)
    e_rho, e_u = errors(got, ref)
    assert e_rho <= 2e-3 and e_u <= 2e-3, (e_rho, e_u)


@pytest.mark.parametrize("case", sorted(GROWING))
def test_step_parity_fp32_growing_regimes(case):
    name, over, spec = GROWING[case]
    model, d = split_preset(name, **over)
    for steps in ((1, 3, 5, 30, 1000) if case == "mips_rho1" else (100, 1000)):
        got = gpu_run(model, d, 64, 64, steps, SEED, spec)
        e, ei = assert_parity(got, model, d, 64, 64, steps, SEED, spec)
        if steps <= 5:
            assert max(e) <= 1e-5, (steps, e)


def _time_average(series, t_from, keys):
    rows = [r for r in series if r["t"] > t_from]
    return {k: np.array([r[k] for r in rows]) for k in keys}


@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
@pytest.mark.parametrize("case", ["cil_rho1_ordered", "passive_noise", "mips_rho1_stable_C"])
def test_16bit_steady_state_observables(storage, case):
    """Where 16-bit rounding decorrelates trajectories, 16-bit storage must
    reproduce the steady-state observables of the FP64 oracle within 1 % or
    3 standard errors (samples every 20 steps after a 1000-step transient)."""
    name, over, spec = (GROWING[case] if case in GROWING else STABLE[case])
    model, d = split_preset(name, **over)
    n, every, steps = 64, 20, 2000
    sim = gpu_sim(model, d, n, n, SEED, spec, storage=storage, sample_every=every, ring=256)
    sim.step(steps)
    gs = sim.observable_series()
    sim.close()
    p = O.params(**d)
    f = O.init(n, n, SEED, **spec, prm=p)
    rs = []
    for k in range(steps // every):
        f = O.run(f, model, p, SEED, k * every, every)
        rs.append(dict(O.observables(f, B=d["B"]), t=(k + 1) * every))
    keys = ("phi", "var_rho", "zeta") if model == "cil" else ("var_rho", "drho_y", "drho_x")
    a, b = _time_average(gs, 1000, keys), _time_average(rs, 1000, keys)
    for k in keys:
        ma, mb = a[k].mean(), b[k].mean()
        se = math.sqrt(a[k].var() / len(a[k]) + b[k].var() / len(b[k])) * 3.0  # samples are correlated: generous
        assert abs(ma - mb) <= max(0.01 * abs(mb), 3 * se), (k, ma, mb, se)


# ------------------------------------------------------ unstable-regime rule
def test_unstable_mips_long_run_statistics():
    """Config 1 with the rescaled MIPS preset at 1000 steps: mass stays within
    the FP32 oracle's own drift and the density variance of the separating
    state agrees with the oracle's within 4x the FP32 oracle's deviation + 5 %."""
    model, d = split_preset("MIPS_RHO1")
    spec = W.INIT_CONFIG1
    steps = 1000
    ref = oracle_run(model, d, 64, 64, steps, SEED, spec)
    f32 = oracle_run(model, d, 64, 64, steps, SEED, spec, bits=32).astype(np.float64)
    got = gpu_run(model, d, 64, 64, steps, SEED, spec)
    m = [O.observables(np.ascontiguousarray(a))["mass"] for a in (got, ref, f32)]
    assert abs(m[0] - m[1]) <= 4 * abs(m[2] - m[1]) + 1e-6 * m[1]
    v = [O.observables(np.ascontiguousarray(a))["var_rho"] for a in (got, ref, f32)]
    assert abs(v[0] - v[1]) <= 4 * abs(v[2] - v[1]) + 0.05 * v[1]


# ------------------------------------------------- ragged sizes and shapes --
SHAPES = [(1, 1), (1, 7), (7, 1), (3, 3), (5, 17), (33, 9), (64, 20), (100, 37), (130, 3), (257, 18)]


@pytest.mark.parametrize("nx,ny", SHAPES)
def test_ragged_sizes_default_shape(nx, ny):
    cases = (("CIL_RHO1", {}, 20, W.init_ordered(U0_CIL)), ("MIPS_RHO1", {}, 3, W.INIT_CONFIG1),
             ("MIPS_RHO1", dict(C=0.2), 40, W.INIT_CONFIG1), ("PASSIVE", dict(sigma=0.01), 40, W.INIT_CONFIG2))
    for name, over, steps, spec in cases:
        model, d = split_preset(name, **over)
        got = gpu_run(model, d, nx, ny, steps, SEED, spec)
        assert_parity(got, model, d, nx, ny, steps, SEED, spec)


SHAPES_FIXED = [(1, 16), (2, 16), (4, 16), (4, 48), (2, 128), (8, 32),
                (1, 16, 4, 3), (2, 32, 2, 4), (4, 64, 4, 6), (2, 48, 4, 3), (8, 32, 2, 4), (4, 16, 1, 3),
                (2, 32, 1, 4), (4, 16, 8, 3), (1, 16, 8, 5), (8, 16, 8, 4), (4, 16, 4, 2), (8, 16, 8, 2),
                (2, 8, 4, 2)]


def staged_refusal(model, storage, shape):
    """Why lbm_set_tuning refuses a staged D2Q9 shape, or None: MIPS needs 3
    row buffers (2 with 16-bit storage, whose MIPS kernel keeps two converted
    FP32 rows per warp), and the buffers must fit a block's 227 KB."""
    if len(shape) < 4:
        return None
    vec, _, warps, stages = shape
    eb = 4 if storage == "f32" else 2
    conv = model == "mips" and eb == 2
    if model == "mips" and stages < (2 if conv else 3):
        return "stages"
    smem = stages * (9 * (warps * 32 * vec + 2 * (16 // eb)) * eb + 16) + (2 * 9 * warps * 32 * vec * 4 if conv else 0)
    return "shared memory" if smem > 232448 else None


@pytest.mark.parametrize("shape", SHAPES_FIXED, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("storage", ["f32", "bf16s"])
@pytest.mark.parametrize("name", ["MIPS_RHO1", "CIL_RHO1", "PASSIVE"])
def test_launch_shapes_give_identical_states(shape, storage, name):
    """Every launch shape -- direct-load (vec, rows) or shared-memory staged
    (vec, rows, warps, stages) -- performs the same per-site arithmetic: the
    states agree bitwise with the (vec 1, rows 16) direct shape, and with the
    oracle."""
    if storage == "f32" and shape[0] == 8:
        pytest.skip("vec 8 is a 16-bit storage shape")
    model, d = split_preset(name, **(dict(sigma=0.01) if name == "PASSIVE" else {}))
    nx, ny = 264, 70
    spec = W.INIT_CONFIG1 if model != "cil" else W.init_ordered(U0_CIL)
    if staged_refusal(model, storage, shape):
        from paper_1902_00530_gb300 import LBMError
        with pytest.raises(LBMError, match="INVALID_ARG"):
            gpu_run(model, d, nx, ny, 9, SEED, spec, storage=storage, tuning=shape)
        return
    base = gpu_run(model, d, nx, ny, 9, SEED, spec, storage=storage, tuning=(1, 16))
    got = gpu_run(model, d, nx, ny, 9, SEED, spec, storage=storage, tuning=shape)
    np.testing.assert_array_equal(got, base)
    if storage == "f32":
        assert_parity(got, model, d, nx, ny, 9, SEED, spec)


@pytest.mark.parametrize("nx,ny", [(4, 4), (8, 3), (36, 5), (64, 64), (96, 33), (520, 17)])
def test_staged_kernel_small_and_ragged(nx, ny):
    """Staged shapes on lattices narrower than a strip, with a ragged last
    strip, and with the periodic halo wrapping onto the strip itself."""
    for name, over, steps, spec in (("MIPS_RHO1", {}, 3, W.INIT_CONFIG1),
                                    ("CIL_RHO1", {}, 20, W.init_ordered(U0_CIL))):
        model, d = split_preset(name, **over)
        for shape in ((1, 16, 4, 3), (4, 32, 2, 4), (4, 16, 8, 3)):
            if nx % shape[0]:
                continue
            got = gpu_run(model, d, nx, ny, steps, SEED, spec, tuning=shape)
            base = gpu_run(model, d, nx, ny, steps, SEED, spec, tuning=(1, 16))
            np.testing.assert_array_equal(got, base)
            assert_parity(got, model, d, nx, ny, steps, SEED, spec)


@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
@pytest.mark.parametrize("nx,ny", [(8, 3), (64, 64), (96, 33), (520, 17)])
def test_staged_mips_16bit_small_and_ragged(nx, ny, storage):
    """The 16-bit MIPS staged kernel, which keeps converted FP32 rows and
    releases each staged row a row early, on lattices narrower than a strip and
    with a ragged last strip (idle lanes and warps), rings of 2 to 4: bitwise
    the direct kernel's states."""
    model, d = split_preset("MIPS_RHO1")
    for shape in ((1, 16, 4, 2), (4, 16, 4, 2), (2, 8, 8, 3), (4, 32, 2, 4), (8, 16, 1, 2)):
        if nx % shape[0]:
            continue
        got = gpu_run(model, d, nx, ny, 5, SEED, W.INIT_CONFIG1, storage=storage, tuning=shape)
        base = gpu_run(model, d, nx, ny, 5, SEED, W.INIT_CONFIG1, storage=storage, tuning=(1, 16))
        np.testing.assert_array_equal(got, base)


# ---------------------------------------------------------- noise stream ---
def _write_state_file(path, f, t, seed, lattice_id, model, storage=0, rho0=1.0):
    """A state file as lbm_save writes it (one lattice): magic, (count, t,
    seed), (nx, ny, storage, model, id, velocity set), rho0, raw populations."""
    q, ny, nx = f.shape
    with open(path, "wb") as fh:
        fh.write(b"LBMSTAT2")
        fh.write(struct.pack("<2qQ", 1, t, seed))
        fh.write(struct.pack("<6i", nx, ny, storage, model, lattice_id, 1 if q == 7 else 0))
        fh.write(struct.pack("<f", rho0))
        fh.write(np.ascontiguousarray(f, dtype=np.float32).tobytes())


@pytest.mark.parametrize("t,lattice_id,seed", [(0, 0, SEED), (7, 3, 12345), (2 ** 31 + 12345, 2 ** 24 - 1,
                                                                                  2 ** 63 + 99)])
def test_noise_stream_matches_oracle(tmp_path, t, lattice_id, seed):
    """Both sides implement Philox4x32-10 and the 14-bit variate recipe from
    the published definition.  From a uniform rest state (a BGK fixed point)
    one step adds exactly the zero-sum noise, which must equal the oracle's
    sigma (s_i - mean s) to FP32 rounding of f (1e-5 here; a wrong bit in the
    top ~15 bits of any variate would exceed it)."""
    from paper_1902_00530_gb300 import Lattice, Simulation
    nx, ny, rho, sigma = 40, 24, 40.0, 0.5
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    f0 = np.broadcast_to((w * rho)[:, None, None], (9, ny, nx)).astype(np.float32)
    path = tmp_path / "rest.lbm"
    _write_state_file(path, f0, t, seed, lattice_id, 0)
    sim = Simulation([Lattice(nx, ny, "f32", lattice_id)], ["passive"], [dict(tau=1.3, sigma=sigma)])
    sim.load(str(path))
    assert sim.time == t
    sim.step(1)
    got = sim.get_state(host=True).numpy().astype(np.float64) - (w * rho)[:, None, None]
    sim.close()
    for (x, y) in [(0, 0), (1, 0), (nx - 1, ny - 1), (17, 5), (3, 20)]:
        s = O.noise_variates(seed, x, y, t, lattice_id)
        eta = sigma * (s - s.mean())
        np.testing.assert_allclose(got[:, y, x], eta, rtol=0, atol=1e-5)


# ------------------------------------------------------------ observables --
def test_sampled_observables_match_oracle():
    """Eq. (phi) and App. D reductions of the stored state every 10 steps."""
    model, d = split_preset("CIL_RHO1")
    nx, ny, every, steps = 96, 40, 10, 60
    spec = W.init_ordered(U0_CIL, rho_amp=0.05, u_amp=0.02)
    sim = gpu_sim(model, d, nx, ny, SEED, spec, sample_every=every, ring=16)
    sim.step(steps)
    series = sim.observable_series()
    now = sim.observables()
    sim.close()
    assert [r["t"] for r in series] == list(range(every, steps + 1, every))
    p = O.params(**d)
    f = O.init(nx, ny, SEED, **spec, prm=p)
    for k, rec in enumerate(series):
        f = O.run(f, model, p, SEED, k * every, every)
        ref = O.observables(f, B=d["B"])
        assert abs(rec["mass"] - ref["mass"]) / ref["mass"] < 1e-6
        for key in ("phi", "drho_y", "drho_x", "zeta"):
            assert abs(rec[key] - ref[key]) < 2e-6, (key, rec[key], ref[key])
        assert abs(rec["var_rho"] - ref["var_rho"]) < 1e-7
    assert now["t"] == steps
    for key in ("mass", "phi", "drho_y", "drho_x", "var_rho", "zeta"):
        assert now[key] == pytest.approx(series[-1][key], rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
def test_sampled_observables_16bit_mips_staged(storage):
    """Sample steps of the 16-bit MIPS staged kernel (converted rows, ring of
    2): the states stay bitwise those of the direct kernel, and every sampled
    record agrees with the direct kernel's to FP32 rounding (the same stored
    values; each thread first sums its vec sites in FP32, so the partial sums
    depend on the launch shape)."""
    model, d = split_preset("MIPS_RHO1")
    nx, ny, every, steps = 264, 70, 3, 12
    runs = []
    for tuning in ((1, 16), (4, 16, 4, 2), (2, 8, 8, 3)):
        sim = gpu_sim(model, d, nx, ny, SEED, W.INIT_CONFIG1, storage=storage, sample_every=every, ring=16,
                      tuning=tuning)
        sim.step(steps)
        runs.append((sim.observable_series(), sim.get_state(host=True).numpy()))
        sim.close()
    (s0, f0) = runs[0]
    assert [r["t"] for r in s0] == list(range(every, steps + 1, every))
    for series, f in runs[1:]:
        np.testing.assert_array_equal(f, f0)
        assert len(series) == len(s0)
        for a, b in zip(series, s0):
            assert a["t"] == b["t"]
            for key in ("mass", "phi", "drho_y", "drho_x", "var_rho", "zeta"):
                assert a[key] == pytest.approx(b[key], rel=1e-6, abs=1e-6), (key, a[key], b[key])


def test_observables_16bit_storage():
    model, d = split_preset("MIPS_PAPER_LITERAL")
    nx, ny = 128, 64
    for storage in ("f16s", "bf16s"):
        sim = gpu_sim(model, d, nx, ny, SEED, W.INIT_CONFIG2, storage=storage)
        sim.step(50)
        ob = sim.observables()
        f = sim.get_state(host=True).numpy().astype(np.float64)
        sim.close()
        ref = O.observables(oracle_run(model, d, nx, ny, 50, SEED, W.INIT_CONFIG2))
        assert abs(ob["mass"] - ref["mass"]) / ref["mass"] < 2e-3
        assert abs(ob["drho_y"] - ref["drho_y"]) < 2e-3 and abs(ob["var_rho"] - ref["var_rho"]) < 2e-3
        # the reduction reads exactly the stored values
        own = O.observables(np.ascontiguousarray(f))
        assert abs(ob["mass"] - own["mass"]) / own["mass"] < 1e-7


@pytest.mark.parametrize("name,over,spec", [("MIPS_RHO1", dict(C=0.2), W.INIT_CONFIG1),
                                             ("CIL_RHO1", {}, W.init_ordered(U0_CIL, u_amp=0.01))])
def test_moments_match_oracle(name, over, spec):
    """lbm_moments against the oracle's moments after 25 steps.  The CIL
    ordered state has a marginal mode (the common direction of u, Sec. 4), so
    rounding differences there do not decay: the bound is 1e-5 or 4x the FP32
    oracle's own divergence, as for the other marginal regimes."""
    model, d = split_preset(name, **over)
    nx, ny = 80, 48
    sim = gpu_sim(model, d, nx, ny, SEED, spec)
    sim.step(25)
    rho, ux, uy = (a.cpu().numpy().astype(np.float64) for a in sim.moments())
    sim.close()
    rr, uxr, uyr = O.moments(oracle_run(model, d, nx, ny, 25, SEED, spec))
    e_rho = np.abs(rho - rr).max()
    e_u = max(np.abs(ux - uxr).max(), np.abs(uy - uyr).max())
    if max(e_rho, e_u) < 1e-5:
        return
    assert name == "CIL_RHO1", (e_rho, e_u)
    r2, ux2, uy2 = O.moments(oracle_run(model, d, nx, ny, 25, SEED, spec, bits=32).astype(np.float64))
    i_rho = np.abs(r2 - rr).max()
    i_u = max(np.abs(ux2 - uxr).max(), np.abs(uy2 - uyr).max())
    assert e_rho <= 4 * i_rho + 1e-6 and e_u <= 4 * i_u + 1e-6, (e_rho, e_u, i_rho, i_u)


@pytest.mark.parametrize("name,over,spec", [("PASSIVE", dict(sigma=0.0099), W.INIT_CONFIG2),
                                             ("MIPS_PAPER_LITERAL", {}, W.INIT_CONFIG2),
                                             ("MIPS_RHO1", {}, W.INIT_CONFIG1)])
def test_mass_conservation_fp32(name, over, spec):
    """Mass over 1000 steps in FP32.  The FP32 sum rho = sum f* that every
    collision conserves is rounded the same way at neighbouring sites whose
    values are nearly equal, so FP32 arithmetic drifts coherently (about 1e-5
    without noise, a few 1e-6 with it, in the FP32 oracle as well).  The GPU
    must stay within 1e-6 or within the FP32 oracle's own drift."""
    model, d = split_preset(name, **over)
    nx, ny = 128, 64
    sim = gpu_sim(model, d, nx, ny, SEED, spec)
    m0 = sim.observables()["mass"]
    sim.step(1000)
    m1 = sim.observables()["mass"]
    sim.close()
    p = O.params(**d)
    f = O.init(nx, ny, SEED, **spec, prm=p, bits=32)
    o0 = O.observables(f)["mass"]
    o1 = O.observables(O.run(f, model, p, SEED, 0, 1000, bits=32))["mass"]
    assert abs(m1 - m0) <= max(abs(o1 - o0), 1e-6 * m0), (m1 - m0, o1 - o0)


# ------------------------------------------------------ bitwise invariants --
@pytest.mark.parametrize("name", ["MIPS_RHO1", "CIL_RHO1"])
def test_density_rescaling_bitwise_gpu(name):
    """(f, C, rho*, A, sigma) -> (2f, C/2, 2rho*, A/4, 2sigma) gives exactly 2x the trajectory."""
    model, d = split_preset(name)
    d2 = dict(d, C=d["C"] / 2, rho_star=d["rho_star"] * 2, A=d["A"] / 4, sigma=d["sigma"] * 2)
    spec = dict(W.INIT_CONFIG2)
    spec2 = dict(spec, rho_mean=2 * spec["rho_mean"])
    a = gpu_run(model, d, 96, 48, 200, SEED, spec)
    b = gpu_run(model, d2, 96, 48, 200, SEED, spec2)
    np.testing.assert_array_equal(b, 2 * a)
    c = gpu_run(model, d2, 96, 48, 200, SEED, spec2, tuning=(2, 32))  # any launch shape
    np.testing.assert_array_equal(c, 2 * a)


def test_batch_equals_solo_runs():
    from paper_1902_00530_gb300 import Lattice, Simulation
    cfg = [(Lattice(64, 64, "f32", 0), "cil", split_preset("CIL_RHO1")[1], W.INIT_CONFIG2),
           (Lattice(96, 32, "f32", 1), "mips", split_preset("MIPS_RHO1")[1], W.INIT_CONFIG1),
           (Lattice(64, 64, "f32", 2), "cil", split_preset("CIL_RHO1", B=0.05)[1], dict(W.INIT_CONFIG2, rho_mean=0.7)),
           (Lattice(128, 40, "bf16s", 3), "mips", split_preset("MIPS_PAPER_LITERAL")[1], W.INIT_CONFIG1)]
    sim = Simulation([c[0] for c in cfg], [c[1] for c in cfg], [c[2] for c in cfg])
    sim.init(SEED, [c[3] for c in cfg])
    sim.step(60)
    batch = [sim.get_state(k, host=True).numpy() for k in range(len(cfg))]
    sim.close()
    for k, (lat, model, d, spec) in enumerate(cfg):
        solo = gpu_run(model, d, lat.nx, lat.ny, 60, SEED, spec, storage=lat.storage, lattice_id=lat.id)
        np.testing.assert_array_equal(batch[k], solo.astype(np.float32))


def test_resume_is_bit_exact(tmp_path):
    model, d = split_preset("MIPS_RHO1")
    sim = gpu_sim(model, d, 64, 48, SEED, W.INIT_CONFIG1)
    sim.step(30)
    sim.save(str(tmp_path / "s.lbm"))
    sim.step(30)
    full = sim.get_state(host=True).numpy()
    sim.close()
    sim = gpu_sim(model, d, 64, 48, SEED + 1, W.INIT_CONFIG2)  # different state, then load
    sim.load(str(tmp_path / "s.lbm"))
    assert sim.time == 30
    sim.step(30)
    np.testing.assert_array_equal(sim.get_state(host=True).numpy(), full)
    sim.close()


@pytest.mark.parametrize("tuning", [None, (2, 32, 4, 0), (2, 32, 4, 4)])
def test_graphs_on_off_identical(tuning):
    model, d = split_preset("MIPS_RHO1")
    a = gpu_run(model, d, 64, 64, 77, SEED, W.INIT_CONFIG2, graphs=True, sample_every=10, ring=8, tuning=tuning)
    b = gpu_run(model, d, 64, 64, 77, SEED, W.INIT_CONFIG2, graphs=False, sample_every=10, ring=8, tuning=tuning)
    np.testing.assert_array_equal(a, b)


def test_parallel_launch_groups_identical():
    """A batch of several launch groups (models, storages and both lattices)
    runs its groups as parallel branches, forked from the bound stream and
    joined before each sample step's finaliser: the states equal those of the
    same batch launched one group after another (per-launch timing on), with
    graphs and without, and so do the sampled records (to FP32 rounding)."""
    from paper_1902_00530_gb300 import Lattice, Simulation
    mips, dm = split_preset("MIPS_RHO1")
    cil, dc = split_preset("CIL_RHO1")
    mips7, dm7 = split_preset("MIPS_Q7_RHO1")
    lats = [Lattice(128, 64, "f32", 0), Lattice(96, 40, "bf16s", 1), Lattice(256, 32, "f32", 2),
            Lattice(64, 64, "f16s", 3), Lattice(128, 48, "f32", 4, "d2q7")]
    mods = [mips, cil, cil, mips, mips7]
    prms = [dm, dc, dc, dm, dm7]
    specs = [W.INIT_CONFIG1, W.init_ordered(U0_CIL), W.init_ordered(U0_CIL), W.INIT_CONFIG1, W.INIT_CONFIG1]
    runs = []
    for graphs, profiling in ((True, False), (False, False), (False, True)):
        sim = Simulation(lats, mods, prms, sample_every=7, ring_capacity=16)
        sim.set_graphs(graphs)
        sim.set_profiling(profiling)
        sim.init(SEED, specs)
        sim.step(30)
        states = [sim.get_state(k, host=True).numpy() for k in range(len(lats))]
        series = [sim.observable_series(k) for k in range(len(lats))]
        sim.close()
        runs.append((states, series))
    for states, series in runs[1:]:
        for a, b in zip(states, runs[0][0]):
            np.testing.assert_array_equal(a, b)
        # each run tunes its own shapes (the joint check of the groups may pick
        # others when timings are close), and a thread's partial sums depend on
        # the shape: records agree to FP32 rounding
        for sa, sb in zip(series, runs[0][1]):
            assert [r["t"] for r in sa] == [r["t"] for r in sb]
            for ra, rb in zip(sa, sb):
                for key in ("mass", "phi", "drho_y", "drho_x", "var_rho", "zeta"):
                    assert ra[key] == pytest.approx(rb[key], rel=1e-6, abs=1e-6), (key, ra[key], rb[key])


def test_rotation_equivariance_gpu():
    """90-degree rotation commutes with the step (sigma = 0), to round-off
    (a linearly stable MIPS setting, so round-off does not grow)."""
    model, d = split_preset("MIPS_RHO1", sigma=0.0, C=0.2)
    n = 64
    from paper_1902_00530_gb300 import Lattice, Simulation
    rot = np.array([0, 2, 3, 4, 1, 6, 7, 8, 5])
    f0 = O.init(n, n, SEED, **W.INIT_CONFIG2, prm=O.params(**d))

    def rotate(f):
        g = np.empty_like(f)
        y, x = np.mgrid[0:n, 0:n]
        for i in range(9):
            g[rot[i], x, (-y) % n] = f[i, y, x]
        return g
    out = []
    for f in (f0, rotate(f0)):
        sim = Simulation([Lattice(n, n)], [model], [d])
        sim.set_state(f.astype(np.float32))
        sim.step(20)
        out.append(sim.get_state(host=True).numpy().astype(np.float64))
        sim.close()
    assert np.abs(rotate(out[0]) - out[1]).max() < 1e-6


# ---------------------------------------------- full size, sampled sites ---
@pytest.mark.parametrize("storage,preset", [("f32", "MIPS_RHO1"), ("bf16s", "MIPS_PAPER_LITERAL"),
                                            ("f16s", "MIPS_PAPER_LITERAL")])
def test_full_size_sampled_parity(storage, preset):
    """The 8192^2 MIPS workload in the tuned launch shape the benchmark uses:
    after k steps, sampled sites (corners, edges, interior) against oracle
    windows of the same global coordinates (exact inside the light cone).
    16-bit storage is checked in the relaxing literal preset."""
    from paper_1902_00530_gb300 import Lattice, Simulation
    model, d = split_preset(preset)
    N, k, R = 8192, 4, 12
    sim = Simulation([Lattice(N, N, storage)], [model], [d])
    sim.init(SEED, [W.INIT_CONFIG1])
    sim.tune()
    sim.step(k)
    rho, ux, uy = (a.cpu().numpy().astype(np.float64) for a in sim.moments())
    sim.close()
    tol = 1e-5 if storage == "f32" else 2e-3
    p = O.params(**d)
    for (cx, cy) in [(0, 0), (N - 1, N - 1), (0, N // 2), (4097, 3), (1234, 5678), (N - 3, 17)]:
        w = 2 * R + 1
        win = (cx - R, cy - R, N, N)
        f = O.run(O.init(w, w, SEED, **W.INIT_CONFIG1, prm=p, window=win), model, p, SEED, 0, k, window=win)
        rr, uxr, uyr = O.moments(f)
        m = R - 2 * k
        ys = [(cy + j) % N for j in range(-m, m + 1)]
        xs = [(cx + i) % N for i in range(-m, m + 1)]
        g_r = rho[np.ix_(ys, xs)]
        sl = slice(R - m, R + m + 1)
        assert np.abs(g_r - rr[sl, sl]).max() / rr.mean() <= tol
        du = max(np.abs(ux[np.ix_(ys, xs)] - uxr[sl, sl]).max(), np.abs(uy[np.ix_(ys, xs)] - uyr[sl, sl]).max())
        assert du / max(np.hypot(uxr, uyr).max(), 1e-3) <= tol


# ------------------------------------------------------------ edge cases ---
def test_zero_steps_and_limits():
    from paper_1902_00530_gb300 import LBMError
    model, d = split_preset("PASSIVE", sigma=0.01)
    sim = gpu_sim(model, d, 16, 16, SEED, W.INIT_CONFIG2)
    f0 = sim.get_state(host=True).numpy()
    sim.step(0)
    assert sim.time == 0
    np.testing.assert_array_equal(sim.get_state(host=True).numpy(), f0)
    with pytest.raises(LBMError):
        sim.step(-1)
    with pytest.raises(LBMError):
        sim.step(2 ** 32)
    with pytest.raises(LBMError):
        sim.observables(lattice=3)
    sim.close()


# --------------------------------------------- sweeps: density and params ---
@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_add_density_matches_oracle(storage):
    """App. C.2: delta rho-bar / Q added to every population mid-run."""
    model, d = split_preset("CIL_PAPER_LITERAL")
    nx, ny, spec = 64, 48, W.INIT_CONFIG2
    sim = gpu_sim(model, d, nx, ny, SEED, spec, storage=storage)
    sim.step(20)
    m0 = sim.observables()["mass"]
    sim.add_density(0.05)
    assert abs(sim.observables()["mass"] - (m0 + 0.05 * nx * ny)) / m0 < 1e-6
    sim.step(20)
    got = sim.get_state(host=True).numpy().astype(np.float64)
    sim.close()
    p = O.params(**d)
    f = O.run(O.init(nx, ny, SEED, **spec, prm=p), model, p, SEED, 0, 20)
    f = O.run(O.add_density(f, 0.05), model, p, SEED, 20, 20)
    tol = 1e-5 if storage == "f32" else 2e-3
    assert max(errors(got, f)) <= tol


def test_set_params_mid_run_matches_oracle():
    """Noise sweep step (App. C.1): sigma changed between steps."""
    model, d = split_preset("MIPS_PAPER_LITERAL")
    d2 = dict(d, sigma=2 * d["sigma"])
    nx, ny, spec = 64, 48, W.INIT_CONFIG1
    sim = gpu_sim(model, d, nx, ny, SEED, spec)
    sim.step(30)
    sim.set_params(d2)
    sim.step(30)
    got = sim.get_state(host=True).numpy().astype(np.float64)
    sim.close()
    p, p2 = O.params(**d), O.params(**d2)
    f = O.run(O.init(nx, ny, SEED, **spec, prm=p), model, p, SEED, 0, 30)
    f = O.run(f, model, p2, SEED, 30, 30)
    assert max(errors(got, f)) <= 1e-5
