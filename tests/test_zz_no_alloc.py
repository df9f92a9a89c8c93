"""The allocation-free observables entry point (lbm_observables_noalloc).

Some callers cannot allocate device memory: code running inside a memory pool
or allocator owned by another runtime, embeddings with a fixed device memory
footprint.  For them the library offers one entry point whose scratch is a
fixed array compiled into the library.  This test calls it through the C ABI
on several states in a row -- so each call runs on scratch the one before left
behind -- and checks each result against the context-based lbm_observables and
the oracle's observables of the same state, within the tolerances the other
observable tests use.  It
lives in its own file, collected last.
"""
import ctypes

import pytest

import workloads as W
from lbmtest import gpu_sim, split_preset

pytestmark = pytest.mark.gpu


def _noalloc(lib, f, B, stream):
    from paper_1902_00530_gb300 import _abi
    o = _abi.lbm_obs()
    st = lib.lbm_observables_noalloc(ctypes.c_void_p(f.data_ptr()), f.shape[2], f.shape[1], B, ctypes.byref(o),
                                     ctypes.c_void_p(stream))
    assert st == 0, st
    return {k: getattr(o, k) for k, _ in _abi.lbm_obs._fields_}


def _close(a, b):
    assert abs(a["mass"] - b["mass"]) / b["mass"] < 1e-6
    for k in ("phi", "drho_y", "drho_x", "zeta"):
        assert abs(a[k] - b[k]) < 2e-6, (k, a[k], b[k])
    assert abs(a["var_rho"] - b["var_rho"]) < 1e-7


def test_noalloc_observables_match_context_and_oracle_twice():
    """Sizes below and above one block's 256 columns and the maximum side (a
    thread then sums several columns), each checked against lbm_observables of
    the same context and the oracle's observables of the same state."""
    import numpy as np
    import oracle as O
    cases = [("CIL_RHO1", 192, 96, W.init_ordered(0.23, rho_amp=0.05, u_amp=0.02)),
             ("MIPS_RHO1", 80, 200, W.INIT_CONFIG1),
             ("CIL_RHO1", 300, 70, W.INIT_CONFIG2),
             ("MIPS_RHO1", 4096, 8, W.INIT_CONFIG1)]
    results = []
    for name, nx, ny, spec in cases:
        model, d = split_preset(name)
        sim = gpu_sim(model, d, nx, ny, W.seed(1), spec)
        sim.step(40)
        ref = sim.observables()
        f = sim.get_state(host=False)          # dense FP32 (9, ny, nx) on the device
        orc = O.observables(f.cpu().numpy().astype(np.float64), B=d["B"])
        results.append((sim, f, d["B"], ref, orc))
    lib = results[0][0].lib
    for sim, f, B, ref, orc in results:        # calls in a row, different sizes
        got = _noalloc(lib, f, B, sim.stream.cuda_stream)
        _close(got, ref)
        _close(got, orc)
    sim, f, B, ref, orc = results[0]           # and the first state again
    _close(_noalloc(lib, f, B, sim.stream.cuda_stream), orc)
    for sim, *_ in results:
        sim.close()


def test_noalloc_rejects_sizes_beyond_the_maximum():
    import torch
    from paper_1902_00530_gb300 import _abi, library
    lib = library()
    f = torch.zeros((9, 1, _abi.NOALLOC_MAX_SIDE + 1), dtype=torch.float32, device="cuda")
    o = _abi.lbm_obs()
    st = lib.lbm_observables_noalloc(ctypes.c_void_p(f.data_ptr()), f.shape[2], 1, 0.0, ctypes.byref(o), None)
    assert st == _abi.LBM_ERR_INVALID_ARG
    st = lib.lbm_observables_noalloc(None, 4, 4, 0.0, ctypes.byref(o), None)
    assert st == _abi.LBM_ERR_INVALID_ARG
