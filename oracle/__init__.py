"""FP64 CPU oracle of the active lattice Boltzmann update (arXiv:1902.00530).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_1902_00530_gb300``) and never imports it.

The arithmetic lives in ``lbm_oracle.c`` (D2Q9) and ``lbm_oracle_d2q7.c``
(the paper's triangular D2Q7 lattice), plain C compiled together with gcc at
``-O2 -ffp-contract=off`` so no fused multiply-adds change its rounding on any
host.  This module only compiles it, loads it with ctypes and moves numpy
arrays in and out.  Populations are numpy arrays of shape (9, ny, nx), or
(7, ny, nx) for the functions with the suffix 7.

Functions and the passages they follow:
  step / run          App. A.2 (steps 1-6), Eq. (fevolution2)
  equilibrium         Eq. (fssD2Q7), D2Q9 form with c_s^2 = 1/3
  negative_correction App. A.3
  gradient            Sec. 3 isotropic stencil, lattice-general form
  ustar               Eqs. (bu_mips), (bu_CIL), (U0) and the U_max clamp
  init                App. C.2 initialisation (f = f^SS of seeded rho, u)
  observables         Eq. (phi); App. D (rho_y std, zeta)
  noise_variates      Eq. (noiseDensityConservation) draws, Philox4x32-10
  *7 (init7, run7, equilibrium7, gradient7, ...)
                      the same on D2Q7: Sec. 2 lattice, Eq. (fssD2Q7) as
                      printed, the Sec. 3 explicit stencils, App. A.3 pairs
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "lbm_oracle_d2q7.c")]
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict[int, ctypes.CDLL] = {}

MODELS = {"passive": 0, "mips": 1, "cil": 2}


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("tau", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("C", ctypes.c_double),
        ("rho_star", ctypes.c_double),
        ("u_max", ctypes.c_double),
        ("A", ctypes.c_double),
        ("B", ctypes.c_double),
    ]


# builds: FP64, FP32, and FP64 with OpenMP row loops (key 65: the same
# arithmetic on several host threads)
_BUILDS = {64: ("double", []), 32: ("float", []), 65: ("double", ["-fopenmp"])}


def _lib_path(bits: int) -> str:
    return os.path.join(_BUILD, f"liblbm_oracle{bits}.so" if bits != 65 else "liblbm_oracle64mt.so")


def build(force: bool = False) -> None:
    """Compile the FP64 and FP32 builds of the oracle, and the FP64 build with
    OpenMP row loops, with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    for bits, (real, extra) in _BUILDS.items():
        out = _lib_path(bits)
        if not force and os.path.exists(out) and all(os.path.getmtime(out) >= os.path.getmtime(src)
                                                     for src in _SRCS):
            continue
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", f"-DREAL={real}", *extra,
               "-o", tmp, *_SRCS, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)


def _key(bits: int, threads: int) -> int:
    if threads == 1:
        return bits
    if bits != 64:
        raise ValueError("the threaded oracle is the FP64 build")
    return 65


def host_cores() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def threads_in_use(threads: int = 0) -> int:
    """Threads the threaded oracle uses; threads > 0 sets the count first
    (0 = all host cores)."""
    lib = _lib(65)
    return int(lib.orc_threads(threads if threads > 0 else host_cores()))


def _lib(bits: int = 64) -> ctypes.CDLL:
    with _LOCK:
        if bits in _LIBS:
            return _LIBS[bits]
        build()
        lib = ctypes.CDLL(_lib_path(bits))
        real_p = ctypes.POINTER(ctypes.c_float if bits == 32 else ctypes.c_double)
        dbl_p = ctypes.POINTER(ctypes.c_double)
        u32, u64, i32, i64 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_int64
        prm = ctypes.POINTER(OrcParams)
        lib.orc_step.argtypes = [real_p, real_p, i32, i32, i32, prm, u64, u32, u32]
        lib.orc_step.restype = i32
        lib.orc_run_window.argtypes = [real_p, i32, i32, i32, prm, u64, u32, i64, u32, i32, i32, i32, i32]
        lib.orc_run_window.restype = i32
        lib.orc_init_window.argtypes = [real_p, i32, i32, u64, u32, ctypes.c_double, ctypes.c_double,
                                        i32, ctypes.c_double, ctypes.c_double, ctypes.c_double, prm,
                                        i32, i32, i32, i32]
        lib.orc_init_window.restype = None
        lib.orc_from_moments.argtypes = [real_p, i32, i32, dbl_p, dbl_p, dbl_p]
        lib.orc_moments.argtypes = [real_p, i32, i32, dbl_p, dbl_p, dbl_p]
        lib.orc_observables.argtypes = [real_p, i32, i32, ctypes.c_double, dbl_p]
        lib.orc_observables.restype = i32
        rl = ctypes.c_float if bits == 32 else ctypes.c_double
        lib.orc_equilibrium.argtypes = [rl] * 3 + [real_p]
        lib.orc_negative_correction.argtypes = [real_p, rl]
        lib.orc_negative_correction.restype = i32
        lib.orc_gradient.argtypes = [real_p, i32, i32, i32, i32, real_p]
        lib.orc_ustar.argtypes = [i32, prm, rl, rl, rl, real_p, real_p]
        lib.orc_philox4x32_10.argtypes = [ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.POINTER(u32)]
        lib.orc_noise_variates.argtypes = [u64, u32, u32, u32, u32, dbl_p]
        lib.orc_init_uniforms.argtypes = [u64, u32, u32, u32, dbl_p]
        lib.orc_real_bytes.restype = i32
        lib.orc7_run_window.argtypes = [real_p, i32, i32, i32, prm, u64, u32, i64, u32, i32, i32, i32, i32]
        lib.orc7_run_window.restype = i32
        lib.orc7_init_window.argtypes = lib.orc_init_window.argtypes
        lib.orc7_init_window.restype = None
        lib.orc7_from_moments.argtypes = [real_p, i32, i32, dbl_p, dbl_p, dbl_p]
        lib.orc7_moments.argtypes = [real_p, i32, i32, dbl_p, dbl_p, dbl_p]
        lib.orc7_observables.argtypes = [real_p, i32, i32, ctypes.c_double, dbl_p]
        lib.orc7_observables.restype = i32
        lib.orc7_equilibrium.argtypes = [rl] * 3 + [real_p]
        lib.orc7_negative_correction.argtypes = [real_p, rl]
        lib.orc7_negative_correction.restype = i32
        lib.orc7_gradient.argtypes = [real_p, i32, i32, i32, i32, real_p]
        lib.orc7_noise_variates.argtypes = [u64, u32, u32, u32, u32, dbl_p]
        ip = ctypes.POINTER(ctypes.c_int)
        lib.orc7_neighbour.argtypes = [i32, i32, i32, i32, i32, i32, ip, ip]
        lib.orc_threads.argtypes = [i32]
        lib.orc_threads.restype = i32
        assert lib.orc_real_bytes() * 8 == (64 if bits == 65 else bits)
        _LIBS[bits] = lib
        return lib


def _dtype(bits: int):
    return np.float32 if bits == 32 else np.float64


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _rp(a: np.ndarray, bits: int):
    return _ptr(a, ctypes.c_float if bits == 32 else ctypes.c_double)


def params(tau=1.0, sigma=0.0, C=0.0, rho_star=1.0, u_max=1.0, A=0.0, B=0.0, **_ignored) -> OrcParams:
    return OrcParams(tau, sigma, C, rho_star, u_max, A, B)


def _check_f(f: np.ndarray, bits: int) -> None:
    if f.ndim != 3 or f.shape[0] != 9:
        raise ValueError("populations must have shape (9, ny, nx)")
    if f.dtype != _dtype(bits) or not f.flags.c_contiguous:
        raise ValueError(f"populations must be C-contiguous {_dtype(bits).__name__}")


def init(nx: int, ny: int, seed: int, lattice_id: int = 0, rho_mean: float = 1.0,
         rho_amp: float = 0.0, u_kind: int = 0, u_amp: float = 0.0, ux0: float = 0.0,
         uy0: float = 0.0, prm: OrcParams | None = None, bits: int = 64, window=None) -> np.ndarray:
    """Seeded initial populations f = f^SS(rho, u) (App. C.2).

    window = (x_off, y_off, gnx, gny): the nx x ny window at that offset of a
    gnx x gny lattice (the draws use the global site coordinates)."""
    lib = _lib(bits)
    f = np.empty((9, ny, nx), dtype=_dtype(bits))
    xo, yo, gx, gy = window if window is not None else (0, 0, nx, ny)
    lib.orc_init_window(_rp(f, bits), nx, ny, seed, lattice_id, rho_mean, rho_amp, u_kind, u_amp,
                        ux0, uy0, ctypes.byref(prm if prm is not None else params()), xo, yo, gx, gy)
    return f


def from_moments(rho: np.ndarray, ux: np.ndarray, uy: np.ndarray, bits: int = 64) -> np.ndarray:
    """f_i = xi_i(rho, u) per site for given (ny, nx) moment fields."""
    lib = _lib(bits)
    rho, ux, uy = (np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy))
    ny, nx = rho.shape
    f = np.empty((9, ny, nx), dtype=_dtype(bits))
    dp = ctypes.POINTER(ctypes.c_double)
    lib.orc_from_moments(_rp(f, bits), nx, ny, _ptr(rho, ctypes.c_double),
                         _ptr(ux, ctypes.c_double), _ptr(uy, ctypes.c_double))
    del dp
    return f


def step(f: np.ndarray, model: str, prm: OrcParams, seed: int, t: int, lattice_id: int = 0,
         bits: int = 64) -> np.ndarray:
    """One step t -> t+1 (App. A.2); returns new populations."""
    _check_f(f, bits)
    lib = _lib(bits)
    out = np.empty_like(f)
    rc = lib.orc_step(_rp(f, bits), _rp(out, bits), f.shape[2], f.shape[1], MODELS[model],
                      ctypes.byref(prm), seed, t, lattice_id)
    if rc != 0:
        raise MemoryError("oracle step failed")
    return out


def run(f: np.ndarray, model: str, prm: OrcParams, seed: int, t0: int, nsteps: int,
        lattice_id: int = 0, bits: int = 64, window=None, threads: int = 1) -> np.ndarray:
    """nsteps steps from t0 (returns a new array; the input is untouched).

    window = (x_off, y_off, gnx, gny) keys the noise by global coordinates; the
    window wraps on itself, so only sites at least nsteps (MIPS: 2 nsteps) from
    its edge are exact.  threads != 1 runs the FP64 step loops on that many
    host threads (0 = all host cores): the same arithmetic, the same result."""
    g = np.array(f, dtype=_dtype(bits), order="C", copy=True)
    _check_f(g, bits)
    lib = _lib(_key(bits, threads))
    if threads != 1:
        threads_in_use(threads)
    xo, yo, gx, gy = window if window is not None else (0, 0, g.shape[2], g.shape[1])
    rc = lib.orc_run_window(_rp(g, bits), g.shape[2], g.shape[1], MODELS[model], ctypes.byref(prm),
                            seed, t0, nsteps, lattice_id, xo, yo, gx, gy)
    if rc != 0:
        raise MemoryError("oracle run failed")
    return g


def add_density(f: np.ndarray, delta_rho_bar: float) -> np.ndarray:
    """App. C.2 density step: add delta / Q to every population (Q = 9)."""
    return f + np.asarray(delta_rho_bar / 9.0, dtype=f.dtype)


def moments(f: np.ndarray, bits: int | None = None):
    """(rho, ux, uy) as float64 (ny, nx) arrays."""
    bits = 64 if f.dtype == np.float64 else 32
    _check_f(f, bits)
    lib = _lib(bits)
    ny, nx = f.shape[1:]
    rho, ux, uy = (np.empty((ny, nx)) for _ in range(3))
    lib.orc_moments(_rp(f, bits), nx, ny, _ptr(rho, ctypes.c_double),
                    _ptr(ux, ctypes.c_double), _ptr(uy, ctypes.c_double))
    return rho, ux, uy


OBS_NAMES = ("mass", "phi", "drho_y", "drho_x", "var_rho", "zeta")


def observables(f: np.ndarray, B: float = 0.0) -> dict:
    """mass, phi (Eq. (phi)), drho_y / drho_x (App. D), var_rho, zeta (App. D)."""
    bits = 64 if f.dtype == np.float64 else 32
    _check_f(f, bits)
    lib = _lib(bits)
    out = np.zeros(6)
    rc = lib.orc_observables(_rp(f, bits), f.shape[2], f.shape[1], B, _ptr(out, ctypes.c_double))
    if rc != 0:
        raise MemoryError("oracle observables failed")
    return dict(zip(OBS_NAMES, out.tolist()))


def equilibrium(rho: float, ux: float, uy: float, bits: int = 64) -> np.ndarray:
    lib = _lib(bits)
    out = np.empty(9, dtype=_dtype(bits))
    lib.orc_equilibrium(rho, ux, uy, _rp(out, bits))
    return out


def negative_correction(f9, rho: float, bits: int = 64):
    """Returns (corrected copy, changed flag) (App. A.3)."""
    lib = _lib(bits)
    g = np.array(f9, dtype=_dtype(bits), copy=True)
    changed = lib.orc_negative_correction(_rp(g, bits), rho)
    return g, bool(changed)


def gradient(rho: np.ndarray, x: int, y: int, bits: int = 64) -> np.ndarray:
    lib = _lib(bits)
    r = np.ascontiguousarray(rho, dtype=_dtype(bits))
    g = np.empty(2, dtype=_dtype(bits))
    lib.orc_gradient(_rp(r, bits), r.shape[1], r.shape[0], x, y, _rp(g, bits))
    return g


def ustar(model: str, prm: OrcParams, rho: float, ux: float, uy: float, g=(0.0, 0.0),
          bits: int = 64) -> np.ndarray:
    lib = _lib(bits)
    ga = np.array(g, dtype=_dtype(bits))
    us = np.empty(2, dtype=_dtype(bits))
    lib.orc_ustar(MODELS[model], ctypes.byref(prm), rho, ux, uy, _rp(ga, bits), _rp(us, bits))
    return us


def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _lib(64)
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def noise_variates(seed: int, x: int, y: int, t: int, lattice_id: int = 0) -> np.ndarray:
    """The nine s_i in (-1, 1) of site (x, y) at step t; eta~_i = sigma s_i."""
    lib = _lib(64)
    s = np.empty(9)
    lib.orc_noise_variates(seed, x, y, t, lattice_id, _ptr(s, ctypes.c_double))
    return s


def init_uniforms(seed: int, x: int, y: int, lattice_id: int = 0) -> np.ndarray:
    lib = _lib(64)
    u = np.empty(4)
    lib.orc_init_uniforms(seed, x, y, lattice_id, _ptr(u, ctypes.c_double))
    return u


# ---------------------------------------------------------------- D2Q7 ----
Q7_E = np.array([[0.0, 0.0]] + [[math.cos(k * math.pi / 3), math.sin(k * math.pi / 3)] for k in range(6)])
Q7_W = np.array([0.5] + [1.0 / 12.0] * 6)


def _check_f7(f: np.ndarray, bits: int) -> None:
    if f.ndim != 3 or f.shape[0] != 7:
        raise ValueError("D2Q7 populations must have shape (7, ny, nx)")
    if f.shape[1] % 2:
        raise ValueError("a periodic D2Q7 box needs an even ny (the odd rows are offset)")
    if f.dtype != _dtype(bits) or not f.flags.c_contiguous:
        raise ValueError(f"populations must be C-contiguous {_dtype(bits).__name__}")


def positions7(nx: int, ny: int):
    """Site positions (X, Y) of the D2Q7 box: X = x + (y mod 2)/2, Y = y sqrt(3)/2."""
    y, x = np.mgrid[0:ny, 0:nx]
    return x + 0.5 * (y % 2), y * (math.sqrt(3.0) / 2.0)


def neighbour7(x: int, y: int, i: int, s: int, nx: int, ny: int):
    """Index of the site at r + s e_i on the D2Q7 box."""
    lib = _lib(64)
    xn, yn = ctypes.c_int(), ctypes.c_int()
    lib.orc7_neighbour(x, y, i, s, nx, ny, ctypes.byref(xn), ctypes.byref(yn))
    return xn.value, yn.value


def init7(nx: int, ny: int, seed: int, lattice_id: int = 0, rho_mean: float = 1.0,
          rho_amp: float = 0.0, u_kind: int = 0, u_amp: float = 0.0, ux0: float = 0.0,
          uy0: float = 0.0, prm: OrcParams | None = None, bits: int = 64, window=None) -> np.ndarray:
    """Seeded D2Q7 initial populations (App. C.2), the same rho, u as init()."""
    if ny % 2:
        raise ValueError("a periodic D2Q7 box needs an even ny")
    lib = _lib(bits)
    f = np.empty((7, ny, nx), dtype=_dtype(bits))
    xo, yo, gx, gy = window if window is not None else (0, 0, nx, ny)
    lib.orc7_init_window(_rp(f, bits), nx, ny, seed, lattice_id, rho_mean, rho_amp, u_kind, u_amp,
                         ux0, uy0, ctypes.byref(prm if prm is not None else params()), xo, yo, gx, gy)
    return f


def from_moments7(rho: np.ndarray, ux: np.ndarray, uy: np.ndarray, bits: int = 64) -> np.ndarray:
    lib = _lib(bits)
    rho, ux, uy = (np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy))
    ny, nx = rho.shape
    f = np.empty((7, ny, nx), dtype=_dtype(bits))
    lib.orc7_from_moments(_rp(f, bits), nx, ny, _ptr(rho, ctypes.c_double),
                          _ptr(ux, ctypes.c_double), _ptr(uy, ctypes.c_double))
    return f


def run7(f: np.ndarray, model: str, prm: OrcParams, seed: int, t0: int, nsteps: int,
         lattice_id: int = 0, bits: int = 64, window=None, threads: int = 1) -> np.ndarray:
    """nsteps D2Q7 steps from t0 (App. A.2); window and threads as in run()
    (the window with an even y offset)."""
    g = np.array(f, dtype=_dtype(bits), order="C", copy=True)
    _check_f7(g, bits)
    lib = _lib(_key(bits, threads))
    if threads != 1:
        threads_in_use(threads)
    xo, yo, gx, gy = window if window is not None else (0, 0, g.shape[2], g.shape[1])
    rc = lib.orc7_run_window(_rp(g, bits), g.shape[2], g.shape[1], MODELS[model], ctypes.byref(prm),
                             seed, t0, nsteps, lattice_id, xo, yo, gx, gy)
    if rc == -2:
        raise ValueError("D2Q7 windows need even ny, y offset and box height")
    if rc != 0:
        raise MemoryError("oracle run failed")
    return g


def add_density7(f: np.ndarray, delta_rho_bar: float) -> np.ndarray:
    """App. C.2 density step on D2Q7: delta / 7 added to every population."""
    return f + np.asarray(delta_rho_bar / 7.0, dtype=f.dtype)


def moments7(f: np.ndarray):
    bits = 64 if f.dtype == np.float64 else 32
    _check_f7(f, bits)
    lib = _lib(bits)
    ny, nx = f.shape[1:]
    rho, ux, uy = (np.empty((ny, nx)) for _ in range(3))
    lib.orc7_moments(_rp(f, bits), nx, ny, _ptr(rho, ctypes.c_double),
                     _ptr(ux, ctypes.c_double), _ptr(uy, ctypes.c_double))
    return rho, ux, uy


def observables7(f: np.ndarray, B: float = 0.0) -> dict:
    bits = 64 if f.dtype == np.float64 else 32
    _check_f7(f, bits)
    lib = _lib(bits)
    out = np.zeros(6)
    rc = lib.orc7_observables(_rp(f, bits), f.shape[2], f.shape[1], B, _ptr(out, ctypes.c_double))
    if rc != 0:
        raise MemoryError("oracle observables failed")
    return dict(zip(OBS_NAMES, out.tolist()))


def equilibrium7(rho: float, ux: float, uy: float, bits: int = 64) -> np.ndarray:
    lib = _lib(bits)
    out = np.empty(7, dtype=_dtype(bits))
    lib.orc7_equilibrium(rho, ux, uy, _rp(out, bits))
    return out


def negative_correction7(f7, rho: float, bits: int = 64):
    lib = _lib(bits)
    g = np.array(f7, dtype=_dtype(bits), copy=True)
    changed = lib.orc7_negative_correction(_rp(g, bits), rho)
    return g, bool(changed)


def gradient7(rho: np.ndarray, x: int, y: int, bits: int = 64) -> np.ndarray:
    lib = _lib(bits)
    r = np.ascontiguousarray(rho, dtype=_dtype(bits))
    g = np.empty(2, dtype=_dtype(bits))
    lib.orc7_gradient(_rp(r, bits), r.shape[1], r.shape[0], x, y, _rp(g, bits))
    return g


def noise_variates7(seed: int, x: int, y: int, t: int, lattice_id: int = 0) -> np.ndarray:
    """The seven s_i in (-1, 1) of a D2Q7 site at step t; eta~_i = sigma s_i."""
    lib = _lib(64)
    s = np.empty(7)
    lib.orc7_noise_variates(seed, x, y, t, lattice_id, _ptr(s, ctypes.c_double))
    return s
