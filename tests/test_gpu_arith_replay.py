"""The FP32 step kernels compute exactly the operation sequence their source
documents, bit for bit: one passive step (noise on and off, tau = 1.3 so that
1/tau and 1 - 1/tau are both inexact, noise strong enough to trigger the App.
A.3 correction at many sites) is replayed here in NumPy float32, one correctly
rounded operation at a time, and compared with the GPU state for a direct and
a staged launch shape.

The replay restates the kernel's arithmetic (collide_v, negative_correction):
pull streaming; rho, j in fixed summation orders; u = j * rcp(rho); the
equilibrium with r = w R folded into each opposite pair, R = rho/tau and the
zero-sum noise shift c folded in when the noise is on; the moving populations
updated as fma(1 - 1/tau, f*, fma(2 sigma, u_i, eq_i)) (noise) or
f* + (eq_i - f*)/tau (no noise); the rest population closed from the mass;
the pairwise correction and the rescale by rho * rcp(sum).  The passive model
is used because its u* needs no reciprocal square root (a hardware
approximation that the CPU cannot reproduce bitwise).  The noise uniforms
come from the oracle's generator, which the noise-stream test pins to the
GPU's.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import workloads as W
from lbmtest import gpu_sim

pytestmark = pytest.mark.gpu

F = np.float32
E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]


def _round32_exact(x: Fraction) -> np.float32:
    """Round an exact rational to the nearest FP32 value, ties to even."""
    r = F(float(x))  # within an ulp; fix by comparing with the neighbours' midpoints
    for _ in range(3):
        lo, hi = np.nextafter(r, F(-np.inf)), np.nextafter(r, F(np.inf))
        mlo = (Fraction(float(lo)) + Fraction(float(r))) / 2
        mhi = (Fraction(float(r)) + Fraction(float(hi))) / 2
        if x < mlo or (x == mlo and (int(np.array(r).view(np.int32)) & 1)):
            r = lo
        elif x > mhi or (x == mhi and (int(np.array(r).view(np.int32)) & 1)):
            r = hi
        else:
            return r
    return r


def fma32(a, b, c):
    """Correctly rounded FP32 a * b + c: the product is exact in FP64; where the
    FP64 sum lies within its own rounding error of an FP32 midpoint, the exact
    rational sum decides."""
    a, b, c = (np.asarray(v, F) for v in np.broadcast_arrays(a, b, c))
    s = a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)
    r = s.astype(F)
    lo, hi = np.nextafter(r, F(-np.inf)), np.nextafter(r, F(np.inf))
    mid_lo = (lo.astype(np.float64) + r.astype(np.float64)) / 2
    mid_hi = (r.astype(np.float64) + hi.astype(np.float64)) / 2
    err = np.spacing(np.abs(s))
    risky = (np.abs(s - mid_lo) <= 2 * err) | (np.abs(s - mid_hi) <= 2 * err)
    for idx in zip(*np.nonzero(risky)):
        exact = Fraction(float(a[idx])) * Fraction(float(b[idx])) + Fraction(float(c[idx]))
        r[idx] = _round32_exact(exact)
    return r


def replay_step(f, tau, sigma, seed, t, lattice_id=0):
    """One passive step of the FP32 kernel, as its source documents it."""
    om = F(1.0 / tau)
    omc = F(1) - om
    ts = F(2.0 * sigma)
    fs = [np.roll(np.roll(f[i], E[i][1], axis=0), E[i][0], axis=1).astype(F) for i in range(9)]
    rho = (((fs[0] + fs[1]) + (fs[2] + fs[3])) + ((fs[4] + fs[5]) + (fs[6] + fs[7]))) + fs[8]
    jx = ((fs[1] + fs[5]) + fs[8]) - ((fs[3] + fs[6]) + fs[7])
    jy = ((fs[2] + fs[5]) + fs[6]) - ((fs[4] + fs[7]) + fs[8])
    inv = np.where(rho > 0, F(1) / rho, F(0)).astype(F)
    sx, sy = jx * inv, jy * inv
    base = fma32(F(-1.5), fma32(sx, sx, sy * sy), F(1))
    noise = sigma > 0
    if noise:
        ny, nx = rho.shape
        u = np.zeros((9, ny, nx), F)
        for y in range(ny):
            for x in range(nx):
                u[:, y, x] = ((O.noise_variates(seed, x, y, t, lattice_id) + 3.0) / 2.0).astype(F)
        su = (((u[0] + u[1]) + (u[2] + u[3])) + ((u[4] + u[5]) + (u[6] + u[7]))) + u[8]
        c = su * (-ts * (F(1) / F(9)))
        R = om * rho
        b1 = fma32((F(1) / F(9)) * R, base, c)
        b5 = fma32((F(1) / F(36)) * R, base, c)
    else:
        R = rho
        b1 = ((F(1) / F(9)) * R) * base
        b5 = ((F(1) / F(36)) * R) * base
    q1, q5 = F(0.5) * R, F(0.125) * R
    k1, k5 = (F(1) / F(3)) * R, (F(1) / F(12)) * R
    p, m = sx + sy, sy - sx
    tx, ty = fma32(q1 * sx, sx, b1), fma32(q1 * sy, sy, b1)
    tp, tm = fma32(q5 * p, p, b5), fma32(q5 * m, m, b5)
    eq = [None, fma32(k1, sx, tx), fma32(k1, sy, ty), fma32(-k1, sx, tx), fma32(-k1, sy, ty),
          fma32(k5, p, tp), fma32(k5, m, tm), fma32(-k5, p, tp), fma32(-k5, m, tm)]
    g = [None] * 9
    for i in range(1, 9):
        g[i] = fma32(omc, fs[i], fma32(ts, u[i], eq[i])) if noise else fma32(om, eq[i] - fs[i], fs[i])
    g[0] = rho - (((g[1] + g[3]) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8])))
    g = np.stack(g).astype(F)
    # App. A.3 at the sites with a negative population (sign bit set)
    neg = (g.view(np.int32) < 0).any(0)
    h = g.copy()
    h[0] = np.maximum(h[0], F(0))
    for a, b in ((1, 3), (2, 4), (5, 7), (6, 8)):
        na = np.minimum(h[a], F(0))
        h[a] = h[a] - na
        h[b] = h[b] - na
        nb = np.minimum(h[b], F(0))
        h[b] = h[b] - nb
        h[a] = h[a] - nb
    s = (((h[0] + h[1]) + (h[2] + h[3])) + ((h[4] + h[5]) + (h[6] + h[7]))) + h[8]
    sc = rho * (F(1) / s)
    h = h * sc
    return np.where(neg[None], h, g).astype(F), int(neg.sum())


@pytest.mark.parametrize("sigma", [0.05, 0.0])
@pytest.mark.parametrize("shape", [(1, 16), (4, 16, 1, 3)], ids=["direct_vec1", "staged_vec4"])
def test_fp32_step_is_its_documented_arithmetic(sigma, shape):
    d = dict(tau=1.3, sigma=sigma)
    nx, ny, seed = 264, 14, W.seed(21)
    sim = gpu_sim("passive", d, nx, ny, seed, dict(W.INIT_CONFIG1, rho_amp=0.05, u_amp=0.02), tuning=shape)
    for t in range(2):
        f = sim.get_state(host=True).numpy().astype(F)
        sim.step(1)
        got = sim.get_state(host=True).numpy().astype(F)
        want, corrected = replay_step(f, 1.3, sigma, seed, t)
        if sigma > 0:
            assert corrected > 100, corrected  # the correction path is exercised
        bad = got != want
        assert not bad.any(), (t, bad.reshape(9, -1).sum(1).tolist())
    sim.close()
