"""ctypes declarations of the C ABI in include/lbm.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbm.so")

LBM_OK, LBM_ERR_INVALID_ARG, LBM_ERR_UNBOUND, LBM_ERR_CUDA = 0, 1, 2, 3
LBM_ERR_TIMEOUT, LBM_ERR_NUMERIC, LBM_ERR_UNSUPPORTED = 4, 5, 6
NOALLOC_MAX_SIDE = 4096
STATUS_NAMES = {0: "LBM_OK", 1: "LBM_ERR_INVALID_ARG", 2: "LBM_ERR_UNBOUND", 3: "LBM_ERR_CUDA",
                4: "LBM_ERR_TIMEOUT", 5: "LBM_ERR_NUMERIC", 6: "LBM_ERR_UNSUPPORTED"}
MODELS = {"passive": 0, "mips": 1, "cil": 2}
STORAGES = {"f32": 0, "f16s": 1, "bf16s": 2}
VELOCITY_SETS = {"d2q9": 0, "d2q7": 1}


class lbm_lattice(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("id", ctypes.c_int32), ("velocity_set", ctypes.c_int32)]


class lbm_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("tau", "sigma", "C", "rho_star", "u_max", "A", "B", "rho0")]


class lbm_init_spec(ctypes.Structure):
    _fields_ = [("rho_mean", ctypes.c_double), ("rho_amp", ctypes.c_double), ("u_kind", ctypes.c_int32),
                ("u_amp", ctypes.c_double), ("ux0", ctypes.c_double), ("uy0", ctypes.c_double)]


class lbm_obs(ctypes.Structure):
    _fields_ = [("t", ctypes.c_int64)] + [(n, ctypes.c_double) for n in
                                          ("mass", "phi", "drho_y", "drho_x", "var_rho", "zeta")]


# name -> (restype, argtypes), in header order
_P = ctypes.c_void_p
_CTX = ctypes.c_void_p
SIGNATURES = {
    "lbm_create": (ctypes.c_int, [ctypes.POINTER(lbm_lattice), ctypes.c_int, ctypes.POINTER(lbm_params),
                                  ctypes.POINTER(_CTX)]),
    "lbm_create_batch": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(lbm_lattice), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(lbm_params), ctypes.POINTER(_CTX)]),
    "lbm_set_sampling": (ctypes.c_int, [_CTX, ctypes.c_int32, ctypes.c_int32]),
    "lbm_buffer_bytes": (ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    "lbm_bind": (ctypes.c_int, [_CTX, _P, _P, _P]),
    "lbm_init": (ctypes.c_int, [_CTX, ctypes.c_uint64, ctypes.POINTER(lbm_init_spec)]),
    "lbm_step": (ctypes.c_int, [_CTX, ctypes.c_int64]),
    "lbm_moments": (ctypes.c_int, [_CTX, ctypes.c_int32, _P, _P, _P]),
    "lbm_observables": (ctypes.c_int, [_CTX, ctypes.c_int32, ctypes.POINTER(lbm_obs)]),
    "lbm_observable_series": (ctypes.c_int, [_CTX, ctypes.c_int32, ctypes.POINTER(lbm_obs), ctypes.c_int32,
                                             ctypes.POINTER(ctypes.c_int32)]),
    "lbm_get_state": (ctypes.c_int, [_CTX, ctypes.c_int32, _P, ctypes.c_int32]),
    "lbm_set_state": (ctypes.c_int, [_CTX, ctypes.c_int32, _P, ctypes.c_int32]),
    "lbm_add_density": (ctypes.c_int, [_CTX, ctypes.c_int32, ctypes.c_double]),
    "lbm_set_params": (ctypes.c_int, [_CTX, ctypes.c_int32, ctypes.POINTER(lbm_params)]),
    "lbm_get_time": (ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_int64)]),
    "lbm_save": (ctypes.c_int, [_CTX, ctypes.c_char_p]),
    "lbm_load": (ctypes.c_int, [_CTX, ctypes.c_char_p]),
    "lbm_set_tuning": (ctypes.c_int, [_CTX, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32]),
    "lbm_tune": (ctypes.c_int, [_CTX]),
    "lbm_get_tuning": (ctypes.c_int, [_CTX, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32)]),
    "lbm_set_graphs": (ctypes.c_int, [_CTX, ctypes.c_int32]),
    "lbm_set_persistent": (ctypes.c_int, [_CTX, ctypes.c_int32, ctypes.c_int32]),
    "lbm_get_persistent": (ctypes.c_int, [_CTX, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "lbm_last_launch_count": (ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_int64)]),
    "lbm_set_profiling": (ctypes.c_int, [_CTX, ctypes.c_int32]),
    "lbm_profile_read": (ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_double)]),
    "lbm_check_wait_timeout": (ctypes.c_int, [_CTX]),
    "lbm_observables_noalloc": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                               ctypes.POINTER(lbm_obs), _P]),
    "lbm_last_error": (ctypes.c_char_p, [_CTX]),
    "lbm_destroy": (None, [_CTX]),
}

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblbm.so; raise if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_1902_00530_gb300.build` "
                           "(the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
