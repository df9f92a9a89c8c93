"""The pins catch plausible mistakes in the oracle.

Each case plants one slip in a temporary copy of the oracle's C source (a
wrong opposite direction, a dropped or mis-signed term, a reversed stream, a
wrong constant...), compiles it, swaps it in for the real oracle and runs a
set of pin tests: at least one must fail.  The committed oracle is never
modified; the planted copies live in a temporary directory.
"""
import ctypes
import os
import subprocess

import pytest

import oracle as O
import test_oracle_pins as P

import test_oracle_d2q7_pins as P7

ODIR = os.path.dirname(O.__file__)
SRCS = {"q9": os.path.join(ODIR, "lbm_oracle.c"), "q7": os.path.join(ODIR, "lbm_oracle_d2q7.c")}

# (name, text in lbm_oracle.c, replacement)
MUTATIONS = [
    ("opposite_table", "static const int OPP[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};",
     "static const int OPP[Q] = {0, 3, 4, 1, 2, 8, 7, 6, 5};"),
    ("equilibrium_quadratic_coefficient", "(real)4.5 * eu * eu", "(real)4.0 * eu * eu"),
    ("equilibrium_linear_sign", "((real)1 + (real)3 * eu", "((real)1 - (real)3 * eu"),
    ("equilibrium_velocity_square", "- (real)1.5 * usq)", "- (real)1.0 * usq)"),
    ("weights_swapped", "if (i <= 4) return (real)1 / (real)9;\n    return (real)1 / (real)36;",
     "if (i <= 4) return (real)1 / (real)36;\n    return (real)1 / (real)9;"),
    ("stream_reversed", "AT(fin, i, wrap(y - EY[i], ny), wrap(x - EX[i], nx))",
     "AT(fin, i, wrap(y + EY[i], ny), wrap(x + EX[i], nx))"),
    ("bgk_times_tau", "f[i] = fi - (fi - feq[i]) / tau;", "f[i] = fi - (fi - feq[i]) * ((real)1 / tau) * ((real)1 / tau);"),
    ("noise_mean_not_removed", "for (int i = 0; i < Q; ++i) f[i] += et[i] - mean;",
     "for (int i = 0; i < Q; ++i) f[i] += et[i];"),
    ("gradient_factor", "g[0] = (real)3 * gx;", "g[0] = (real)2 * gx;"),
    ("gradient_y_sign", "gy += weight(i) * r * (real)EY[i];", "gy -= weight(i) * r * (real)EY[i];"),
    ("mips_ceiling_inverted", "if (rho < rs) {", "if (rho > rs) {"),
    ("cil_u0_linear", "real a_rho2 = (real)p->A * rho * rho;", "real a_rho2 = (real)p->A * rho;"),
    ("correction_no_rescale", "for (int i = 0; i < Q; ++i) f[i] = f[i] * (rho / sum);", "(void)sum;"),
    ("correction_not_moved", "f[OPP[i]] += -f[i];", "(void)OPP;"),
    ("phi_not_normalised", "out[1] = sqrt(px * px + py * py) / m;", "out[1] = sqrt(px * px + py * py);"),
    ("column_std_over_rows", "double d = col[x] / ny - mean;", "double d = col[x] / nx - mean;"),
    ("noise_variance", "s[i] = (2.0 * (double)m[i] + 1.0 - 16384.0) / 16384.0;",
     "s[i] = (2.0 * (double)m[i] + 1.0 - 16384.0) / 32768.0;"),
    ("clamp_ignored", "if (mag > (real)p->u_max) {", "if (mag > (real)1e30) {"),
    ("philox_round_multiplier", "#define PHILOX_M0 0xD2511F53u", "#define PHILOX_M0 0xD2511F55u"),
    ("philox_key_increment", "#define PHILOX_W1 0xBB67AE85u", "#define PHILOX_W1 0xBB67AE87u"),
    # the window form: noise keyed by window instead of global coordinates, the
    # offset applied with the wrong sign, init draws at window coordinates
    ("window_noise_at_window_coordinates",
     "orc_noise_variates(seed, (uint32_t)wrap(x + x_off, gnx), (uint32_t)wrap(y + y_off, gny),",
     "orc_noise_variates(seed, (uint32_t)x, (uint32_t)y,"),
    ("window_offset_sign",
     "orc_noise_variates(seed, (uint32_t)wrap(x + x_off, gnx), (uint32_t)wrap(y + y_off, gny),",
     "orc_noise_variates(seed, (uint32_t)wrap(x - x_off, gnx), (uint32_t)wrap(y - y_off, gny),"),
    ("window_init_at_window_coordinates",
     "orc_init_uniforms(seed, (uint32_t)wrap(x + x_off, gnx), (uint32_t)wrap(y + y_off, gny), id,",
     "orc_init_uniforms(seed, (uint32_t)x, (uint32_t)y, id,"),
]

# slips in the D2Q7 file: (name, text in lbm_oracle_d2q7.c, replacement)
MUTATIONS7 = [
    ("q7_row_offset_sign", "int twice_x = 2 * x + par_y + s * E2X[i];", "int twice_x = 2 * x - par_y + s * E2X[i];"),
    ("q7_stream_reversed", "orc7_neighbour(x, y, i, -1, nx, ny, &xs, &ys);",
     "orc7_neighbour(x, y, i, +1, nx, ny, &xs, &ys);"),
    ("q7_opposite_table", "static const int OPP7[Q7] = {0, 4, 5, 6, 1, 2, 3};",
     "static const int OPP7[Q7] = {0, 4, 6, 5, 1, 3, 2};"),
    ("q7_equilibrium_quadratic", "(real)8 * eu * eu", "(real)4.5 * eu * eu"),
    ("q7_equilibrium_velocity_square", "- (real)2 * usq)", "- (real)1.5 * usq)"),
    ("q7_weights", "return i == 0 ? (real)1 / (real)2 : (real)1 / (real)12;",
     "return i == 0 ? (real)4 / (real)10 : (real)1 / (real)10;"),
    ("q7_row_spacing", "return (real)ERY[i] * (real)sqrt(3.0) / (real)2;", "return (real)ERY[i];"),
    ("q7_gradient_dy", "((real)4 * dy)", "((real)4 * dx)"),
    ("q7_gradient_x_terms", "(r[2] + r[6]) - (r[3] + r[5])", "(r[2] + r[3]) - (r[5] + r[6])"),
    ("q7_noise_mean_over_nine", "mean = mean / (real)Q7;", "mean = mean / (real)9;"),
    ("q7_init_row_spacing", "double eu = 0.5 * E2X[i] * vx + hs3 * ERY[i] * vy;",
     "double eu = 0.5 * E2X[i] * vx + 0.5 * ERY[i] * vy;"),
    ("q7_moments_row_spacing", "jy += fi * hs3 * ERY[i];", "jy += fi * 0.5 * ERY[i];"),
    ("q7_noise_bits", "s[i] = (2.0 * (double)h + 1.0 - 65536.0) / 65536.0;",
     "s[i] = (2.0 * (double)h + 1.0 - 65536.0) / 131072.0;"),
    ("q7_window_noise_at_window_coordinates",
     "orc7_noise_variates(seed, (uint32_t)wrap7(x + x_off, gnx), (uint32_t)wrap7(y + y_off, gny), t, id,",
     "orc7_noise_variates(seed, (uint32_t)x, (uint32_t)y, t, id,"),
    ("q7_window_offset_sign",
     "orc7_noise_variates(seed, (uint32_t)wrap7(x + x_off, gnx), (uint32_t)wrap7(y + y_off, gny), t, id,",
     "orc7_noise_variates(seed, (uint32_t)wrap7(x - x_off, gnx), (uint32_t)wrap7(y - y_off, gny), t, id,"),
    ("q7_window_init_at_window_coordinates",
     "orc_init_uniforms(seed, (uint32_t)wrap7(x + x_off, gnx), (uint32_t)wrap7(y + y_off, gny), id, U);",
     "orc_init_uniforms(seed, (uint32_t)x, (uint32_t)y, id, U);"),
]

# the pin checks run against each planted copy (all fast)
PINS = [
    (P.test_equilibrium_moments_textbook_d2q9, {}),
    (P.test_equilibrium_at_rest_is_weights, {}),
    (P.test_negative_correction_bruteforce, {}),
    (P.test_negative_correction_examples, {}),
    (P.test_gradient_stencil_single_mode, dict(n=16, m=1)),
    (P.test_ustar_closures, {}),
    (P.test_mass_conservation, dict(name="MIPS_RHO1")),
    (P.test_fixed_points, dict(case="passive_u")),
    (P.test_homogeneous_relaxation_closed_forms, dict(tau=1.5)),
    (P.test_passive_shear_wave_viscosity, dict(tau=1.0)),
    (P.test_mips_growth_rate_matches_chapman_enskog, dict(tau=1.5, C=0.2)),
    (P.test_cil_growth_rate_matches_banding_condition, dict(A=0.4, B=0.5)),
    (P.test_rotation_equivariance, dict(name="MIPS_RHO1")),
    (P.test_observables_closed_forms, {}),
    (P.test_noise_statistics, {}),
    (P.test_philox_matches_an_independent_library_implementation, {}),
    (P.test_window_equals_interior_of_periodic_run, dict(name="MIPS_RHO1", reach=2)),
]


PINS7 = [
    (P7.test_neighbours_follow_positions, dict(nx=5, ny=4)),
    (P7.test_streaming_moves_populations_along_e, {}),
    (P7.test_equilibrium_moments_textbook_d2q7, {}),
    (P7.test_equilibrium_at_rest_is_weights7, {}),
    (P7.test_negative_correction_bruteforce7, {}),
    (P7.test_negative_correction_examples7, {}),
    (P7.test_gradient_stencils_on_plane_waves, dict(nx=9, ny=14, m=2, n=3)),
    (P7.test_mass_conservation7, dict(name="MIPS_RHO1")),
    (P7.test_passive_shear_wave_viscosity7, dict(axis="y", tau=1.0)),
    (P7.test_passive_shear_wave_viscosity7, dict(axis="x", tau=1.0)),
    (P7.test_mips_growth_rate_matches_chapman_enskog7, dict(axis="y", tau=1.0, C=1.0)),
    (P7.test_noise_statistics7, {}),
    (P7.test_init7_recipe, {}),
    (P7.test_window_equals_interior_of_periodic_run7, dict(name="MIPS_RHO1", reach=2)),
]


def _build(tmp_path, name, old, new, which):
    srcs = []
    for key, path in SRCS.items():
        text = open(path).read()
        if key == which:
            assert old in text, f"mutation site of {name} not found in the oracle"
            text = text.replace(old, new, 1)
        src = tmp_path / f"{name}_{key}.c"
        src.write_text(text)
        srcs.append(str(src))
    libs = {}
    for bits, real in ((64, "double"), (32, "float")):
        out = tmp_path / f"{name}{bits}.so"
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", f"-DREAL={real}", "-o", str(out),
                        *srcs, "-lm"], check=True)
        libs[bits] = str(out)
    return libs


CASES = [(m, "q9") for m in MUTATIONS] + [(m, "q7") for m in MUTATIONS7]


@pytest.mark.parametrize("mut,which", CASES, ids=[m[0] for m, _ in CASES])
def test_pins_catch_planted_mistake(tmp_path, monkeypatch, mut, which):
    name, old, new = mut
    libs = _build(tmp_path, name, old, new, which)
    O._lib(64)
    O._lib(32)
    saved = dict(O._LIBS)
    caught = []
    try:
        for bits in (64, 32):
            O._LIBS.pop(bits, None)
        monkeypatch.setattr(O, "_lib_path", lambda bits: libs[bits])
        monkeypatch.setattr(O, "build", lambda force=False: None)
        for fn, kw in (PINS if which == "q9" else PINS7):
            try:
                fn(**kw)
            except AssertionError:
                caught.append(fn.__name__)
    finally:
        O._LIBS.clear()
        O._LIBS.update(saved)
    assert caught, f"no pin caught the planted mistake {name}"
