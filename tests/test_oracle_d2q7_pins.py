"""Pins of the D2Q7 (triangular lattice) oracle to what the paper and the
mathematics fix.

The lattice geometry is pinned against positions computed here from the
paper's e_i (Sec. 2) and the brick box, not against the oracle's own offset
arithmetic; the equilibrium against its textbook moments with c_s^2 = 1/4;
the explicit Sec. 3 stencils against the vector form a sum (rho_i - rho_i+3) e_i
on plane waves; the whole update against Chapman-Enskog viscosities and
growth rates (App. B) in both lattice directions, the Sec. 7 noise moment
<h_x h_x> = c^2 sigma^2, exact symmetries and conservation laws.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

S3 = math.sqrt(3.0)
E = O.Q7_E
EX7, EY7 = E[:, 0], E[:, 1]
CS2 = 0.25


def prm_of(name, **kw):
    d = W.preset(name, **kw)
    return d.pop("model"), O.params(**d)


def _pos(x, y):
    return x + 0.5 * (y % 2), y * S3 / 2


def _site_at(X, Y, nx, ny):
    """Index of the site at point (X, Y) of the periodic brick box (None if no site)."""
    yf = Y / (S3 / 2)
    y = int(round(yf))
    if abs(yf - y) > 1e-9:
        return None
    xf = X - 0.5 * (y % 2)
    x = int(round(xf))
    if abs(xf - x) > 1e-9:
        return None
    return x % nx, y % ny


# ------------------------------------------------------------ geometry ----
def test_velocity_set_is_the_papers():
    """Sec. 2: unit vectors 60 degrees apart (the only reading under which the
    Sec. 3 stencils hold), opposite pairs 1-4, 2-5, 3-6 (App. A.3)."""
    assert np.allclose(np.hypot(EX7[1:], EY7[1:]), 1.0)
    for i in range(1, 7):
        j = (i + 2) % 6 + 1
        assert np.allclose(E[j], -E[i])
    assert abs(sum(E[1:, 0])) < 1e-15 and abs(sum(E[1:, 1])) < 1e-15


@pytest.mark.parametrize("nx,ny", [(8, 6), (5, 4), (1, 2), (3, 2)])
def test_neighbours_follow_positions(nx, ny):
    """The oracle's r + s e_i is the site at position r + s e_i of the box."""
    for y in range(ny):
        for x in range(nx):
            X, Y = _pos(x, y)
            for i in range(7):
                for s in (1, -1):
                    want = _site_at(X + s * EX7[i], Y + s * EY7[i], nx, ny)
                    assert O.neighbour7(x, y, i, s, nx, ny) == want, (x, y, i, s)


def test_streaming_moves_populations_along_e():
    """With 1/tau ~ 0 and no noise the update is the streaming of App. A.2 step
    1: f_i arrives at the site at r + e_i (positions computed here)."""
    nx, ny = 6, 8
    rng = np.random.default_rng(4)
    f = rng.uniform(0.05, 0.2, (7, ny, nx))
    g = O.run7(f, "passive", O.params(tau=1e15), 1, 0, 1)
    for y in range(ny):
        for x in range(nx):
            X, Y = _pos(x, y)
            for i in range(7):
                xn, yn = _site_at(X + EX7[i], Y + EY7[i], nx, ny)
                assert abs(g[i, yn, xn] - f[i, y, x]) < 1e-14


# --------------------------------------------------------- equilibrium ----
def test_equilibrium_moments_textbook_d2q7():
    """Eq. (fssD2Q7): sum xi = rho, sum xi e = rho u, sum xi e e = rho (I/4 + u u)
    and sum xi e_a e_b e_c = (rho/4)(u_a d_bc + u_b d_ac + u_c d_ab) (c_s^2 = 1/4)."""
    rng = np.random.default_rng(1)
    for _ in range(200):
        rho = rng.uniform(0.1, 3.0)
        u = rng.uniform(-0.2, 0.2, 2)
        xi = O.equilibrium7(rho, u[0], u[1])
        assert abs(xi.sum() - rho) <= 1e-14 * rho
        np.testing.assert_allclose(xi @ E, rho * u, rtol=0, atol=1e-14)
        P = np.einsum("i,ia,ib->ab", xi, E, E)
        np.testing.assert_allclose(P, rho * (CS2 * np.eye(2) + np.outer(u, u)), rtol=0, atol=1e-14)
        T = np.einsum("i,ia,ib,ic->abc", xi, E, E, E)
        d = np.eye(2)
        want = rho * CS2 * (np.einsum("a,bc->abc", u, d) + np.einsum("b,ac->abc", u, d)
                            + np.einsum("c,ab->abc", u, d))
        np.testing.assert_allclose(T, want, rtol=0, atol=1e-14)


def test_equilibrium_at_rest_is_weights7():
    np.testing.assert_allclose(O.equilibrium7(2.0, 0.0, 0.0), 2.0 * O.Q7_W, rtol=1e-15)


# ---------------------------------------------------- negative correction --
OPP = np.array([0, 4, 5, 6, 1, 2, 3])


def test_negative_correction_bruteforce7():
    rng = np.random.default_rng(2)
    for trial in range(3000):
        f = rng.uniform(-0.05, 0.3, 7)
        if trial % 3 == 0:
            i = int(rng.integers(1, 4))
            f[i] = -rng.uniform(0, 0.05)
            f[OPP[i]] = -rng.uniform(0, 0.05)
        rho = max(f.sum(), 1e-3)
        g, changed = O.negative_correction7(f, rho)
        assert (g >= 0).all()
        if not changed:
            np.testing.assert_array_equal(g, f)
            continue
        assert abs(g.sum() - rho) <= 1e-14 * max(rho, 1)
        j_in, j = f @ E, g @ E
        assert abs(j[0] * j_in[1] - j[1] * j_in[0]) <= 1e-13
        if np.abs(j_in).sum() > 1e-6:
            assert j @ j_in > 0


def test_negative_correction_examples7():
    """Worked cases of App. A.3 with the pairs 1<->4, 2<->5, 3<->6."""
    f = np.array([0.4, 0.1, -0.02, 0.1, 0.1, 0.1, 0.1])
    g, _ = O.negative_correction7(f, 0.88)
    h = f.copy(); h[5] += 0.02; h[2] = 0.0
    np.testing.assert_allclose(g, h * (0.88 / h.sum()), rtol=1e-15)
    f = np.array([0.4, 0.1, 0.1, -0.01, 0.1, 0.1, -0.03])  # 3 <-> 6 both negative
    g, _ = O.negative_correction7(f, 0.76)
    h = f.copy(); h[6] += 0.01; h[3] = 0.0; h[3] += -h[6]; h[6] = 0.0
    np.testing.assert_allclose(g, h * (0.76 / h.sum()), rtol=1e-14)


# ------------------------------------------------------------ gradient ----
@pytest.mark.parametrize("nx,ny,m,n", [(12, 8, 1, 1), (9, 14, 2, 3), (20, 6, 3, 0), (7, 10, 0, 2)])
def test_gradient_stencils_on_plane_waves(nx, ny, m, n):
    """rho = a + b sin(k.R) with k periodic on the box: the Sec. 3 explicit
    stencils equal the vector form (1/3) sum_{i=1..3} (rho_i - rho_{i+3}) e_i
    = (2b/3) cos(k.R) sum_{i=1..3} sin(k.e_i) e_i at every site."""
    a, b = 1.0, 0.1
    k = np.array([2 * np.pi * m / nx, 2 * np.pi * n / (ny * S3 / 2)])
    X, Y = O.positions7(nx, ny)
    rho = a + b * np.sin(k[0] * X + k[1] * Y)
    for y in range(ny):
        for x in range(nx):
            ph = k[0] * X[y, x] + k[1] * Y[y, x]
            want = (2 * b / 3) * math.cos(ph) * sum(math.sin(k @ E[i]) * E[i] for i in (1, 2, 3))
            np.testing.assert_allclose(O.gradient7(rho, x, y), want, rtol=0, atol=1e-14)


def test_gradient_is_isotropic_to_second_order():
    """For long waves the stencil is the gradient in every direction, with an
    error O(k^3) (the isotropy the paper asks of it, Sec. 3)."""
    errs = []
    for L in (60, 120):
        nx, ny = L, 2 * L
        X, Y = O.positions7(nx, ny)
        for (m, n) in ((1, 0), (0, 1), (1, 1)):
            k = np.array([2 * np.pi * m / nx, 2 * np.pi * n / (ny * S3 / 2)])
            rho = 1 + 0.1 * np.sin(k[0] * X + k[1] * Y)
            g = O.gradient7(rho, 3, 5)
            want = 0.1 * math.cos(k[0] * X[5, 3] + k[1] * Y[5, 3]) * k
            errs.append(np.abs(g - want).max() / (0.1 * np.linalg.norm(k) ** 3))
    assert max(errs) < 0.2


# --------------------------------------------------------- conservation ----
@pytest.mark.parametrize("name", ["MIPS_RHO1", "CIL_RHO1", "MIPS_PAPER_LITERAL", "PASSIVE"])
def test_mass_conservation7(name):
    model, p = prm_of(name)
    if name == "PASSIVE":
        p.sigma = 0.02
    f = O.init7(30, 24, W.seed(1), **W.INIT_CONFIG2, prm=p)
    m0 = O.observables7(f)["mass"]
    g = O.run7(f, model, p, W.seed(1), 0, 600)
    assert abs(O.observables7(g)["mass"] - m0) / m0 < 1e-13


@pytest.mark.parametrize("case", ["passive_u", "cil_U0", "mips_rest"])
def test_fixed_points7(case):
    n = 10
    rho = np.full((n, n), 1.1)
    if case == "passive_u":
        model, p, u = "passive", O.params(tau=1.3), (0.03, -0.02)
    elif case == "cil_U0":
        p = O.params(tau=1.7, A=0.1, B=0.3)
        U0 = 0.3 - 0.1 * 1.1 ** 2
        model, u = "cil", (U0 * 0.6, U0 * 0.8)
    else:
        model, p, u = "mips", O.params(tau=1.2, C=6, rho_star=5 / 3, u_max=0.3), (0.0, 0.0)
    f = O.from_moments7(rho, np.full((n, n), u[0]), np.full((n, n), u[1]))
    g = O.run7(f, model, p, 5, 0, 500)
    np.testing.assert_allclose(g, f, rtol=0, atol=1e-14)


@pytest.mark.parametrize("tau", [1.0, 1.6])
def test_homogeneous_relaxation_closed_forms7(tau):
    n = 6
    rho = np.full((n, n), 0.9)
    u0 = np.array([0.05, 0.12])
    f = O.from_moments7(rho, np.full((n, n), u0[0]), np.full((n, n), u0[1]))
    lam = 1 - 1 / tau
    for nsteps in (1, 4):
        _, ux, uy = O.moments7(O.run7(f, "mips", O.params(tau=tau, C=6, rho_star=5 / 3, u_max=0.3), 1, 0, nsteps))
        np.testing.assert_allclose([ux[3, 4], uy[3, 4]], lam ** nsteps * u0, atol=1e-14)
        U0 = 0.3 - 0.1 * 0.81
        _, ux, uy = O.moments7(O.run7(f, "cil", O.params(tau=tau, A=0.1, B=0.3), 1, 0, nsteps))
        mag = math.hypot(ux[2, 5], uy[2, 5])
        assert abs((mag - U0) - lam ** nsteps * (np.linalg.norm(u0) - U0)) < 1e-14


# ------------------------------------------------- Chapman-Enskog (App. B) --
@pytest.mark.parametrize("axis", ["y", "x"])
@pytest.mark.parametrize("tau", [0.8, 1.0, 1.7])
def test_passive_shear_wave_viscosity7(axis, tau):
    """Passive limit, nu = (2 tau - 1) c_s^2 / 2 = (tau - 1/2)/4 on D2Q7 (App. B:
    c_s = c/2).  A shear wave across the rows (u_x(Y)) and one along them
    (u_y(X), X including the half-site offset of the odd rows)."""
    U = 1e-4
    if axis == "y":
        nx, ny = 2, 128
        X, Y = O.positions7(nx, ny)
        k = 2 * np.pi / (ny * S3 / 2)
        ph = k * Y
        ux, uy = U * np.sin(ph), np.zeros_like(ph)
    else:
        nx, ny = 128, 2
        X, Y = O.positions7(nx, ny)
        k = 2 * np.pi / nx
        ph = k * X
        ux, uy = np.zeros_like(ph), U * np.sin(ph)
    f = O.from_moments7(np.ones_like(ph), ux, uy)
    p = O.params(tau=tau)
    t1, t2 = 50, 650
    g1 = O.run7(f, "passive", p, 1, 0, t1)
    g2 = O.run7(g1, "passive", p, 1, t1, t2 - t1)
    comp = 1 if axis == "y" else 2
    a = [abs(np.sum(O.moments7(g)[comp] * np.sin(ph))) for g in (g1, g2)]
    nu = (tau - 0.5) / 4
    nu_meas = -math.log(a[1] / a[0]) / ((t2 - t1) * k * k)
    assert abs(nu_meas - nu) / nu < 2e-3


def _growth_rate7(model, p, u0, L, axis):
    if axis == "x":
        nx, ny = L, 2
        X, Y = O.positions7(nx, ny)
        k = 2 * np.pi / nx
        ph = k * X
        ub = (u0, 0.0)
    else:
        nx, ny = 2, L
        X, Y = O.positions7(nx, ny)
        k = 2 * np.pi / (ny * S3 / 2)
        ph = k * Y
        ub = (0.0, u0)
    rho = 1 + 1e-6 * np.cos(ph)
    f = O.from_moments7(rho, np.full(ph.shape, ub[0]), np.full(ph.shape, ub[1]))

    def amp(g):
        r = O.moments7(g)[0]
        return abs(np.sum((r - r.mean()) * np.exp(-1j * ph)))

    g1 = O.run7(f, model, p, 1, 0, 20)
    g2 = O.run7(g1, model, p, 1, 20, 80)
    return math.log(amp(g2) / amp(g1)) / 80, k


@pytest.mark.parametrize("axis", ["x", "y"])
@pytest.mark.parametrize("tau,C", [(1.0, 0.0), (1.5, 0.2), (1.0, 1.0)])
def test_mips_growth_rate_matches_chapman_enskog7(axis, tau, C):
    """App. B with the D2Q7 pressure c_s^2 rho = rho/4:
    s = -k^2 (c_s^2 - gamma rho0 C (1 - rho0/rho*)) / gamma, gamma = 2/(2 tau - 1),
    approached as O(k^2); along x and across the rows."""
    p = O.params(tau=tau, C=C, rho_star=5 / 3, u_max=0.3)
    gam = 2 / (2 * tau - 1)
    errs = []
    for L in (128, 256):
        s, k = _growth_rate7("mips", p, 0.0, L, axis)
        ce = -k * k * (CS2 - gam * C * (1 - 0.6)) / gam
        errs.append(abs(s - ce) / abs(ce))
    assert errs[0] < 4e-3 and errs[1] < 1.2e-3
    assert errs[1] < errs[0] / 2.5 or errs[1] < 1e-6


@pytest.mark.parametrize("axis", ["x", "y"])
@pytest.mark.parametrize("A,B", [(0.06845, 0.3), (0.4, 0.5)])
def test_cil_growth_rate_matches_banding_condition7(axis, A, B):
    """Sec. 6 banding condition with the D2Q7 c_s^2 = 1/4:
    Re s = k^2 (2 tau - 1)(U0'^2 rho0^2 - c_s^2)/2 for a wave along the flow."""
    p = O.params(tau=1.0, A=A, B=B)
    U0, dU0 = B - A, -2 * A
    errs = []
    for L in (128, 256):
        s, k = _growth_rate7("cil", p, U0, L, axis)
        ce = k * k * (dU0 ** 2 - CS2) / 2
        errs.append(abs(s - ce) / abs(ce))
    assert errs[0] < 4e-3 and errs[1] < 1.2e-3
    assert errs[1] < errs[0] / 2.5 or errs[1] < 1e-6


# ---------------------------------------------------------- symmetries ----
def _mirror_x(f):
    """X -> -X: site (x, y) -> (-x - (y mod 2)) mod nx; e1<->e4, e2<->e3, e5<->e6."""
    perm = [0, 4, 3, 2, 1, 6, 5]
    _, ny, nx = f.shape
    g = np.empty_like(f)
    for y in range(ny):
        xs = (-np.arange(nx) - (y % 2)) % nx
        for i in range(7):
            g[perm[i], y, xs] = f[i, y, :]
    return g


def _mirror_y(f):
    """Y -> -Y (ny even keeps the row parity): e2<->e6, e3<->e5."""
    perm = [0, 1, 6, 5, 4, 3, 2]
    _, ny, nx = f.shape
    g = np.empty_like(f)
    for y in range(ny):
        for i in range(7):
            g[perm[i], (-y) % ny, :] = f[i, y, :]
    return g


def test_mirror_tables_match_velocity_set():
    for perm, flip in (([0, 4, 3, 2, 1, 6, 5], (-1, 1)), ([0, 1, 6, 5, 4, 3, 2], (1, -1))):
        for i in range(7):
            assert np.allclose(E[perm[i]], E[i] * np.array(flip))


@pytest.mark.parametrize("name", ["MIPS_RHO1", "CIL_RHO1"])
@pytest.mark.parametrize("mirror", [_mirror_x, _mirror_y])
def test_reflection_equivariance7(name, mirror):
    model, p = prm_of(name, sigma=0.0)
    f = O.init7(12, 10, 4, **W.INIT_CONFIG2, prm=p)
    np.testing.assert_allclose(mirror(O.run7(f, model, p, 4, 0, 15)), O.run7(mirror(f), model, p, 4, 0, 15),
                               rtol=0, atol=1e-12)


@pytest.mark.parametrize("name", ["MIPS_RHO1", "CIL_RHO1"])
@pytest.mark.parametrize("bits", [64, 32])
def test_density_rescaling_symmetry_bitwise7(name, bits):
    d = W.preset(name)
    model = d.pop("model")
    p1 = O.params(**d)
    p2 = O.params(**dict(d, C=d["C"] / 2, rho_star=d["rho_star"] * 2, A=d["A"] / 4, sigma=d["sigma"] * 2))
    f = O.init7(14, 10, 77, **W.INIT_CONFIG2, prm=p1, bits=bits)
    g1 = O.run7(f, model, p1, 77, 0, 40, bits=bits)
    g2 = O.run7(2 * f, model, p2, 77, 0, 40, bits=bits)
    np.testing.assert_array_equal(g2, 2 * g1)


# --------------------------------------------------------------- noise ----
def test_noise_statistics7():
    """eta~ uniform on [-sigma, sigma] (Sec. 2), and the Sec. 7 moment of
    h = sum eta_i c e_i: <h_x h_x> = <h_y h_y> = c^2 sigma^2, <h_x h_y> = 0."""
    n = 40000
    s = np.array([O.noise_variates7(W.seed(1), i % 200, i // 200, 17) for i in range(n)])
    assert np.all(np.abs(s) < 1)
    assert np.all(np.abs(s.mean(0)) < 5 * math.sqrt(1 / 3 / n))
    assert np.all(np.abs(s.var(0) - 1 / 3) < 5 * math.sqrt(4 / 45 / n))
    assert np.abs(np.corrcoef(s.T) - np.eye(7)).max() < 5 / math.sqrt(n)
    eta = s - s.mean(1, keepdims=True)  # sigma = 1
    h = eta @ E
    assert abs(h[:, 0].var() - 1.0) < 5 * math.sqrt(2 / n)
    assert abs(h[:, 1].var() - 1.0) < 5 * math.sqrt(2 / n)
    assert abs(np.mean(h[:, 0] * h[:, 1])) < 5 / math.sqrt(n)
    k = s * 2 ** 16  # 16-bit grid: odd multiples of 2^-16
    assert np.all(k == np.round(k)) and np.all(np.round(k) % 2 == 1)
    assert not np.array_equal(O.noise_variates7(1, 3, 4, 5), O.noise_variates7(1, 3, 4, 6))


# --------------------------------------------------------- observables ----
def test_observables_closed_forms7():
    """Eq. (phi) and App. D on D2Q7 states.  A density cosine along X averages
    over a column whose sites alternate between X = x and x + 1/2, so
    rho_y(x) has amplitude a cos(pi / (2 nx)) and drho_y = a cos(pi/(2 nx)) / sqrt 2."""
    nx, ny = 24, 16
    X, Y = O.positions7(nx, ny)
    f = O.from_moments7(np.full((ny, nx), 1.2), np.full((ny, nx), 0.03), np.full((ny, nx), -0.04))
    ob = O.observables7(f, B=0.3)
    assert abs(ob["phi"] - 0.05) < 1e-14 and abs(ob["zeta"] - 0.25) < 1e-14
    assert abs(ob["mass"] - 1.2 * nx * ny) < 1e-14 * 1.2 * nx * ny
    a = 0.07
    f = O.from_moments7(1 + a * np.cos(2 * np.pi * X / nx), np.zeros((ny, nx)), np.zeros((ny, nx)))
    ob = O.observables7(f, B=0.3)
    assert abs(ob["drho_y"] - a * math.cos(math.pi / (2 * nx)) / math.sqrt(2)) < 1e-14
    assert ob["drho_x"] < 1e-12 and abs(ob["var_rho"] - a * a / 2) < 1e-14
    b = 0.05
    f = O.from_moments7(1 + b * np.sin(2 * np.pi * 2 * Y / (ny * S3 / 2)), np.zeros((ny, nx)), np.zeros((ny, nx)))
    ob = O.observables7(f, B=0.3)
    assert abs(ob["drho_x"] - b / math.sqrt(2)) < 1e-14 and ob["drho_y"] < 1e-12


def test_d2q7_box_needs_even_rows():
    with pytest.raises(ValueError):
        O.init7(8, 5, 1)
    f = O.init7(8, 6, 1)
    with pytest.raises(ValueError):
        O.run7(f, "passive", O.params(), 1, 0, 1, window=(0, 1, 8, 6))


def test_init7_recipe():
    """App. C.2 on D2Q7: the moments of the initial state are the seeded rho and
    u (uniforms from the pinned Philox draws) for each u_kind."""
    p = O.params(A=0.06845, B=0.3)
    nx, ny = 9, 6
    for spec in (dict(rho_mean=1.0, rho_amp=0.1, u_kind=0, u_amp=0.02, ux0=0.01, uy0=-0.005),
                 dict(rho_mean=0.8, rho_amp=0.05, u_kind=1, u_amp=0.03, ux0=0.0, uy0=0.01),
                 dict(rho_mean=1.0, rho_amp=0.1, u_kind=2, u_amp=0.0, ux0=0.0, uy0=0.0)):
        f = O.init7(nx, ny, 5, lattice_id=3, **spec, prm=p)
        rho, ux, uy = O.moments7(f)
        for y in range(ny):
            for x in range(nx):
                U = O.init_uniforms(5, x, y, 3)
                r = spec["rho_mean"] * (1 + spec["rho_amp"] * (2 * U[0] - 1))
                if spec["u_kind"] == 0:
                    u = (spec["ux0"] + spec["u_amp"] * (2 * U[1] - 1), spec["uy0"] + spec["u_amp"] * (2 * U[2] - 1))
                elif spec["u_kind"] == 1:
                    a = 2 * math.pi * U[1]
                    u = (spec["ux0"] + spec["u_amp"] * math.cos(a), spec["uy0"] + spec["u_amp"] * math.sin(a))
                else:
                    a = 2 * math.pi * U[1]
                    U0 = max(0.3 - 0.06845 * r * r, 0.0)
                    u = (U0 * math.cos(a), U0 * math.sin(a))
                assert abs(rho[y, x] - r) < 1e-14
                assert abs(ux[y, x] - u[0]) < 1e-14 and abs(uy[y, x] - u[1]) < 1e-14


# ------------------------------------------------------------ windows ----
WINDOWS7 = [(30, 28, 24, 20), (5, 2, 18, 16), (0, 30, 40, 12)]  # even y offsets and heights, 40 x 36 box


def _window_of7(full, x_off, y_off, nx, ny):
    gny, gnx = full.shape[1:]
    ys = (y_off + np.arange(ny)) % gny
    xs = (x_off + np.arange(nx)) % gnx
    return full[:, ys][:, :, xs]


@pytest.mark.parametrize("name,reach", [("MIPS_RHO1", 2), ("CIL_RHO1", 1)])
def test_window_equals_interior_of_periodic_run7(name, reach):
    """The D2Q7 window form against the full periodic box: equal everywhere at
    init and, after k noisy steps, inside the light cone (a hop moves at most
    one row and one column on the brick box; MIPS's gradient adds one hop)."""
    model, p = prm_of(name)
    gnx, gny, seed, k = 40, 36, 7654321, 3
    full0 = O.init7(gnx, gny, seed, **W.INIT_CONFIG2, prm=p)
    full = O.run7(full0, model, p, seed, 9, k)
    for (xo, yo, nx, ny) in WINDOWS7:
        win = (xo, yo, gnx, gny)
        w0 = O.init7(nx, ny, seed, **W.INIT_CONFIG2, prm=p, window=win)
        np.testing.assert_array_equal(w0, _window_of7(full0, xo, yo, nx, ny))
        wk = O.run7(w0, model, p, seed, 9, k, window=win)
        ref = _window_of7(full, xo, yo, nx, ny)
        m = reach * k
        inner_x = slice(m, nx - m) if nx < gnx else slice(None)
        np.testing.assert_array_equal(wk[:, m:ny - m, inner_x], ref[:, m:ny - m, inner_x])
        assert not np.array_equal(wk[:, :m], ref[:, :m])
