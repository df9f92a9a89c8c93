"""C-ABI checks that need no GPU: the library builds, loads, exports every
symbol include/lbm.h declares, and validates arguments on the host."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1902_00530_gb300 import _abi
    from paper_1902_00530_gb300.build import build
    build()
    return _abi.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", text)))


def test_header_declares_the_calls():
    names = declared_symbols()
    for required in ("lbm_create", "lbm_init", "lbm_step", "lbm_moments", "lbm_observables",
                     "lbm_create_batch", "lbm_bind", "lbm_buffer_bytes", "lbm_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1902_00530_gb300 import _abi
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert name in _abi.SIGNATURES, f"binding lacks {name}"


def _lat(nx=8, ny=8, storage=0, id_=0, vs=0):
    from paper_1902_00530_gb300 import _abi
    return _abi.lbm_lattice(nx, ny, storage, id_, vs)


def _prm(**kw):
    from paper_1902_00530_gb300 import _params
    return _params(kw)


@pytest.mark.parametrize("bad", [
    dict(lat=dict(nx=0)), dict(lat=dict(ny=70000)), dict(lat=dict(storage=3)), dict(lat=dict(id_=1 << 24)),
    dict(prm=dict(tau=0.5)), dict(prm=dict(sigma=-1.0)), dict(prm=dict(tau=float("nan"))),
    dict(model=7), dict(model=1, prm=dict(rho_star=0.0)), dict(prm=dict(rho0=-1.0)),
    dict(prm=dict(A=float("inf")), model=2),
    dict(lat=dict(vs=2)), dict(lat=dict(vs=1, ny=7)),  # unknown velocity set; D2Q7 with odd ny
])
def test_create_rejects_bad_arguments(lib, bad):
    ctx = ctypes.c_void_p(123)
    lat = _lat(**bad.get("lat", {}))
    prm = _prm(**{"tau": 1.0, **bad.get("prm", {})})
    st = lib.lbm_create(ctypes.byref(lat), bad.get("model", 0), ctypes.byref(prm), ctypes.byref(ctx))
    assert st == 1 and not ctx.value


def test_host_only_calls_and_status_codes(lib):
    ctx = ctypes.c_void_p()
    lat = _lat(37, 5)
    prm = _prm(tau=1.0, sigma=0.01)
    assert lib.lbm_create(ctypes.byref(lat), 0, ctypes.byref(prm), ctypes.byref(ctx)) == 0
    sb, cb = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.lbm_buffer_bytes(ctx, ctypes.byref(sb), ctypes.byref(cb)) == 0
    # two FP32 buffers of 9 planes, rows padded to 128 bytes
    assert sb.value >= 2 * 9 * 5 * 64 * 4 and cb.value > 0
    assert lib.lbm_set_sampling(ctx, 10, 0) == 1          # sampling needs a ring
    assert lib.lbm_set_sampling(ctx, 10, 8) == 0
    sb2 = ctypes.c_size_t()
    assert lib.lbm_buffer_bytes(ctx, ctypes.byref(sb2), ctypes.byref(cb)) == 0
    assert lib.lbm_step(ctx, 1) == 2                      # not bound
    assert b"bound" in lib.lbm_last_error(ctx)
    assert lib.lbm_observables(ctx, 0, None) == 2
    assert lib.lbm_set_tuning(ctx, 1, 4, 32, 4, 0) == 1   # 4 does not divide 37
    assert lib.lbm_set_tuning(ctx, 1, 1, 4, 4, 0) == 1    # rows below 8
    assert lib.lbm_set_tuning(ctx, 1, 1, 32, 9, 0) == 1   # too many warps
    assert lib.lbm_set_tuning(ctx, 1, 1, 32, 2, 3) == 1   # staged needs nx % 4 == 0 (37)
    assert lib.lbm_set_tuning(ctx, 1, 1, 32, 2, 0) == 0
    v, r, w, s = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    args = [ctypes.byref(x) for x in (v, r, w, s)]
    assert lib.lbm_get_tuning(ctx, 0, *args) == 0
    assert (v.value, r.value, w.value, s.value) == (1, 32, 2, 0)
    assert lib.lbm_get_tuning(ctx, 1, *args) == 1
    t = ctypes.c_int64(-1)
    assert lib.lbm_get_time(ctx, ctypes.byref(t)) == 0 and t.value == 0
    assert lib.lbm_check_wait_timeout(ctx) == 2            # the failure-path check needs bound buffers
    assert lib.lbm_set_persistent(None, 1, 0) == 1
    assert lib.lbm_set_persistent(ctx, 1, -1) == 1         # lattice-group budget out of range
    assert lib.lbm_set_persistent(ctx, 1, (1 << 20) + 1) == 1
    assert lib.lbm_set_persistent(ctx, 3, 0) == 1          # modes are 0, 1, 2
    on = ctypes.c_int32(-1)
    assert lib.lbm_get_persistent(ctx, 0, ctypes.byref(on)) == 0 and on.value == 0  # default 2: not tuned yet
    assert lib.lbm_set_persistent(ctx, 1, 0) == 0          # host only before binding
    assert lib.lbm_get_persistent(ctx, 0, ctypes.byref(on)) == 0 and on.value == 1  # direct D2Q9 shape
    assert lib.lbm_set_tuning(ctx, 1, 4, 16, 2, 0) == 1 and lib.lbm_set_tuning(ctx, 1, 1, 32, 2, 0) == 0
    assert lib.lbm_get_persistent(ctx, 1, ctypes.byref(on)) == 1   # no lattice 1
    assert lib.lbm_get_persistent(ctx, 0, None) == 1
    assert lib.lbm_set_persistent(ctx, 2, 64) == 0
    assert lib.lbm_set_persistent(ctx, 0, 16) == 0
    assert lib.lbm_get_persistent(ctx, 0, ctypes.byref(on)) == 0 and on.value == 0
    assert lib.lbm_bind(ctx, None, None, None) == 1
    assert lib.lbm_bind(ctx, ctypes.c_void_p(0x1001), ctypes.c_void_p(0x2000), None) == 1  # misaligned
    lib.lbm_destroy(ctx)
    lib.lbm_destroy(None)


def test_staged_block_width_limits(lib):
    """Staged blocks of both velocity sets take 1..8 warps (the warps share each
    staged row); 9 is refused."""
    from paper_1902_00530_gb300 import _abi
    prm = _prm(tau=1.0, sigma=0.01)
    for vs in (0, 1):
        ctx = ctypes.c_void_p()
        lat = _abi.lbm_lattice(64, 32, 0, 0, vs)
        assert lib.lbm_create(ctypes.byref(lat), 0, ctypes.byref(prm), ctypes.byref(ctx)) == 0
        assert lib.lbm_set_tuning(ctx, 1, 1, 16, 8, 3) == 0
        assert lib.lbm_set_tuning(ctx, 1, 1, 16, 4, 3) == 0
        assert lib.lbm_set_tuning(ctx, 1, 1, 16, 9, 3) == 1
        lib.lbm_destroy(ctx)


def test_mips_ring_depth(lib):
    """A staged MIPS ring holds its density halo: 3 row buffers at least with
    FP32 storage, 2 with 16-bit storage (whose kernel keeps the rows it has
    converted); the other closures take 2."""
    from paper_1902_00530_gb300 import _abi
    for model, storage, least in ((1, 0, 3), (1, 1, 2), (1, 2, 2), (2, 0, 2), (0, 1, 2)):
        prm = _prm(tau=1.0, sigma=0.01, C=6.0, rho_star=5.0 / 3.0, u_max=0.3, A=0.06845, B=0.3)
        ctx = ctypes.c_void_p()
        lat = _abi.lbm_lattice(256, 64, storage, 0)
        assert lib.lbm_create(ctypes.byref(lat), model, ctypes.byref(prm), ctypes.byref(ctx)) == 0
        for stages in (2, 3):
            assert lib.lbm_set_tuning(ctx, 1, 4, 16, 4, stages) == (0 if stages >= least else 1), (model, storage)
        lib.lbm_destroy(ctx)


def test_staged_shared_memory_limit(lib):
    """A staged shape whose row buffers exceed the 227 KB of shared memory a
    block can have is refused when it is set, not at launch: D2Q9 FP32 with 8
    warps of vec 4 takes 37 168 B per buffer, so 6 buffers fit and 7 do not;
    the D2Q7 buffer (28 912 B) fits 8."""
    from paper_1902_00530_gb300 import _abi
    prm = _prm(tau=1.0, sigma=0.01)
    for vs, fits in ((0, 6), (1, 8)):
        ctx = ctypes.c_void_p()
        lat = _abi.lbm_lattice(1024, 64, 0, 0, vs)
        assert lib.lbm_create(ctypes.byref(lat), 0, ctypes.byref(prm), ctypes.byref(ctx)) == 0
        for stages in range(2, 9):
            assert lib.lbm_set_tuning(ctx, 1, 4, 16, 8, stages) == (0 if stages <= fits else 1), (vs, stages)
        lib.lbm_destroy(ctx)


def test_batch_create_groups(lib):
    from paper_1902_00530_gb300 import _abi
    n = 4
    lats = (_abi.lbm_lattice * n)(*[_abi.lbm_lattice(64, 32, s, k) for k, s in enumerate([0, 1, 0, 2])])
    mods = (ctypes.c_int * n)(1, 2, 1, 2)
    prms = (_abi.lbm_params * n)(*[_prm(tau=1.0, rho_star=2.0) for _ in range(n)])
    ctx = ctypes.c_void_p()
    assert lib.lbm_create_batch(n, lats, mods, prms, ctypes.byref(ctx)) == 0
    sb, cb = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.lbm_buffer_bytes(ctx, ctypes.byref(sb), ctypes.byref(cb)) == 0
    # 2 f32 + 2 16-bit lattices, two buffers each
    assert sb.value >= 2 * 9 * 32 * (2 * 64 * 4 + 2 * 64 * 2)
    lib.lbm_destroy(ctx)
    assert lib.lbm_create_batch(0, lats, mods, prms, ctypes.byref(ctx)) == 1


def test_python_binding_refuses_without_library(tmp_path):
    from paper_1902_00530_gb300 import _abi
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _abi._lib_saved = _abi._lib
        try:
            _abi._lib = None
            _abi.load(str(tmp_path / "missing.so"))
        finally:
            _abi._lib = _abi._lib_saved


def test_d2q7_buffers_and_tuning(lib):
    """A D2Q7 lattice holds seven planes per buffer; its strips need an even
    number of rows; staged shapes apply to both lattices."""
    from paper_1902_00530_gb300 import _abi
    lats = (_abi.lbm_lattice * 2)(_abi.lbm_lattice(64, 30, 0, 0, 1), _abi.lbm_lattice(64, 30, 0, 1, 0))
    mods = (ctypes.c_int * 2)(2, 2)
    prms = (_abi.lbm_params * 2)(*[_prm(tau=1.0, A=0.06845, B=0.3) for _ in range(2)])
    ctx = ctypes.c_void_p()
    assert lib.lbm_create_batch(2, lats, mods, prms, ctypes.byref(ctx)) == 0
    sb = ctypes.c_size_t(); cb = ctypes.c_size_t()
    assert lib.lbm_buffer_bytes(ctx, ctypes.byref(sb), ctypes.byref(cb)) == 0
    plane = 30 * 64 * 4
    assert 2 * (7 + 9) * plane <= sb.value < 2 * (7 + 9) * plane + 4 * 256
    assert lib.lbm_set_tuning(ctx, 1, 2, 17, 4, 0) == 1   # odd rows: D2Q7 needs even
    assert lib.lbm_set_tuning(ctx, 1, 2, 32, 2, 3) == 0
    v, r, w, st = (ctypes.c_int32() for _ in range(4))
    assert lib.lbm_get_tuning(ctx, 0, *[ctypes.byref(x) for x in (v, r, w, st)]) == 0
    assert (v.value, r.value, st.value) == (2, 32, 3)
    assert lib.lbm_get_tuning(ctx, 1, *[ctypes.byref(x) for x in (v, r, w, st)]) == 0
    assert st.value == 3
    lib.lbm_destroy(ctx)


def test_direct_kernel_index_limit(lib):
    """The direct D2Q9 kernel indexes a buffer with 32-bit element offsets: a
    lattice of more than 2^32 elements per buffer (9 ny pitch) starts on a
    staged shape and refuses direct ones; one that cannot be staged either (nx
    not a multiple of 16 bytes) is refused at create.  D2Q7 is not limited.
    Host only: nothing is allocated."""
    from paper_1902_00530_gb300 import _abi
    prm = _prm(tau=1.0, C=6.0, rho_star=1.6, u_max=0.3, sigma=0.08)
    v, r, w, st = (ctypes.c_int32() for _ in range(4))

    def create(nx, ny, storage=0, vs=0):
        ctx = ctypes.c_void_p()
        status = lib.lbm_create(ctypes.byref(_abi.lbm_lattice(nx, ny, storage, 0, vs)), 1, ctypes.byref(prm),
                                ctypes.byref(ctx))
        return status, ctx

    # 9 * 14563 * 32768 = 4294803456 <= 2^32: direct shapes allowed
    status, ctx = create(32768, 14563)
    assert status == 0
    assert lib.lbm_get_tuning(ctx, 0, *[ctypes.byref(x) for x in (v, r, w, st)]) == 0 and st.value == 0
    assert lib.lbm_set_tuning(ctx, 1, 4, 32, 4, 0) == 0
    lib.lbm_destroy(ctx)
    # one row more crosses 2^32: staged by default, direct refused, staged accepted
    status, ctx = create(32768, 14564)
    assert status == 0
    assert lib.lbm_get_tuning(ctx, 0, *[ctypes.byref(x) for x in (v, r, w, st)]) == 0 and st.value == 4
    assert lib.lbm_set_tuning(ctx, 1, 4, 32, 4, 0) == 1
    assert lib.lbm_set_tuning(ctx, 1, 4, 32, 4, 3) == 0
    lib.lbm_destroy(ctx)
    # FP16 storage: pitch in 64-element steps; nx = 65530 pads to 65536 and is not a
    # multiple of 8 elements, so it can be neither direct nor staged at this height
    assert create(65530, 8000, storage=1)[0] == 6
    assert create(65530, 7000, storage=1)[0] == 0     # 9 * 7000 * 65536 < 2^32
    status, ctx = create(65530, 8000, storage=1, vs=1)  # D2Q7 keeps 64-bit indexing
    assert status == 0
    lib.lbm_destroy(ctx)


def test_binding_names_the_unsupported_lattice(lib):
    """The Python binding reports LBM_ERR_UNSUPPORTED with its reason before
    touching the GPU (creation is host only)."""
    from paper_1902_00530_gb300 import LBMError, Lattice, Simulation
    with pytest.raises(LBMError) as e:
        Simulation([Lattice(65530, 8000, "f16s")], ["mips"], [dict(tau=1.0, C=6.0, rho_star=1.6, u_max=0.3)])
    assert e.value.status == 6 and "staged kernel" in str(e.value)


def test_persistent_applies_to_direct_shapes_of_both_lattices(lib):
    """lbm_get_persistent under mode 1: groups on a direct kernel (D2Q9 and
    the paper's D2Q7) take persistent launches, staged groups do not; mode 0
    turns them off and mode 2 waits for the tuner.  Host only, no GPU."""
    from paper_1902_00530_gb300 import _abi
    on = ctypes.c_int32(-1)
    for vs, ny in ((0, 16), (1, 16)):
        ctx = ctypes.c_void_p()
        lat = _lat(64, ny, 0, 0, vs)
        prm = _prm(tau=1.0, sigma=0.01, A=0.068, B=0.3)
        assert lib.lbm_create(ctypes.byref(lat), _abi.MODELS["cil"], ctypes.byref(prm), ctypes.byref(ctx)) == 0
        assert lib.lbm_set_persistent(ctx, 1, 0) == 0
        assert lib.lbm_set_tuning(ctx, 1, 2, 8, 4, 0) == 0          # direct
        assert lib.lbm_get_persistent(ctx, 0, ctypes.byref(on)) == 0 and on.value == 1
        assert lib.lbm_set_tuning(ctx, 1, 2, 8, 4, 3) == 0          # staged
        assert lib.lbm_get_persistent(ctx, 0, ctypes.byref(on)) == 0 and on.value == 0
        assert lib.lbm_set_tuning(ctx, 1, 2, 8, 4, 0) == 0
        assert lib.lbm_set_persistent(ctx, 2, 0) == 0               # the tuner has not chosen yet
        assert lib.lbm_get_persistent(ctx, 0, ctypes.byref(on)) == 0 and on.value == 0
        assert lib.lbm_set_persistent(ctx, 0, 0) == 0
        assert lib.lbm_get_persistent(ctx, 0, ctypes.byref(on)) == 0 and on.value == 0
        lib.lbm_destroy(ctx)
