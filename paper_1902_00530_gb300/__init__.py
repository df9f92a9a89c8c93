"""GB300-native active lattice Boltzmann (Nesbitt, Pruessner & Lee, arXiv:1902.00530).

A thin Python binding over the C ABI of ``liblbm.so`` (``include/lbm.h``).
Every step of the method runs in the library's CUDA kernels; this module only
marshals arguments.  PyTorch supplies the device buffers and the stream.

    sim = Simulation([Lattice(1024, 1024)], ["cil"], [dict(tau=1, sigma=0.05, A=0.068, B=0.3)])
    sim.init(seed=1, specs=[dict(rho_mean=1, rho_amp=0.1, u_kind=1, u_amp=0.01)])
    sim.step(1000)
    rho, ux, uy = sim.moments()
    print(sim.observables())
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

from . import _abi

__all__ = ["Lattice", "Simulation", "LBMError", "build", "library"]


class LBMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_abi.STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


@dataclass
class Lattice:
    nx: int
    ny: int
    storage: str = "f32"          # "f32", "f16s" or "bf16s"
    id: int = 0                   # random-stream id
    velocity_set: str = "d2q9"    # "d2q9", or "d2q7" (the paper's triangular lattice; ny even)

    @property
    def q(self) -> int:
        return 7 if self.velocity_set == "d2q7" else 9


def build(force: bool = False) -> str:
    from .build import build as _build
    return _build(force=force)


def library():
    return _abi.load()


_PARAM_KEYS = ("tau", "sigma", "C", "rho_star", "u_max", "A", "B", "rho0")
_SPEC_KEYS = ("rho_mean", "rho_amp", "u_kind", "u_amp", "ux0", "uy0")


def _params(d: dict) -> _abi.lbm_params:
    base = dict(tau=1.0, sigma=0.0, C=0.0, rho_star=1.0, u_max=1.0, A=0.0, B=0.0, rho0=0.0)
    base.update({k: v for k, v in d.items() if k in _PARAM_KEYS})
    return _abi.lbm_params(*[float(base[k]) for k in _PARAM_KEYS])


def _spec(d: dict) -> _abi.lbm_init_spec:
    s = dict(rho_mean=1.0, rho_amp=0.0, u_kind=0, u_amp=0.0, ux0=0.0, uy0=0.0)
    s.update({k: v for k, v in d.items() if k in _SPEC_KEYS})
    return _abi.lbm_init_spec(float(s["rho_mean"]), float(s["rho_amp"]), int(s["u_kind"]),
                              float(s["u_amp"]), float(s["ux0"]), float(s["uy0"]))


class Simulation:
    """One context: a single lattice or a batch advanced together."""

    def __init__(self, lattices, models, params, sample_every: int = 0, ring_capacity: int = 0,
                 device=None, stream=None):
        import torch
        self._torch = torch
        self.lib = _abi.load()
        if isinstance(lattices, Lattice):
            lattices, models, params = [lattices], [models], [params]
        n = len(lattices)
        if not (len(models) == len(params) == n) or n < 1:
            raise ValueError("lattices, models and params need the same non-zero length")
        self.lattices = list(lattices)
        self.models = [m if isinstance(m, str) else {0: "passive", 1: "mips", 2: "cil"}[m] for m in models]
        lats = (_abi.lbm_lattice * n)(*[_abi.lbm_lattice(l.nx, l.ny, _abi.STORAGES[l.storage], l.id,
                                                         _abi.VELOCITY_SETS[l.velocity_set])
                                        for l in lattices])
        mods = (ctypes.c_int * n)(*[_abi.MODELS[m] for m in self.models])
        prms = (_abi.lbm_params * n)(*[_params(p) for p in params])
        ctx = ctypes.c_void_p()
        st = self.lib.lbm_create_batch(n, lats, mods, prms, ctypes.byref(ctx))
        if st == _abi.LBM_ERR_UNSUPPORTED:
            raise LBMError(st, "a D2Q9 lattice beyond 2^32 elements per buffer runs only the staged kernel, "
                               "which needs nx a multiple of 16 bytes of storage")
        if st != 0:
            raise LBMError(st, "invalid lattice or parameters")
        self.ctx = ctx
        self._check(self.lib.lbm_set_sampling(self.ctx, int(sample_every), int(ring_capacity)))
        sb, cb = ctypes.c_size_t(), ctypes.c_size_t()
        self._check(self.lib.lbm_buffer_bytes(self.ctx, ctypes.byref(sb), ctypes.byref(cb)))
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        self.state = torch.empty(max(sb.value, 256), dtype=torch.uint8, device=self.device)
        self.scratch = torch.empty(max(cb.value, 256), dtype=torch.uint8, device=self.device)
        self._check(self.lib.lbm_bind(self.ctx, self.state.data_ptr(), self.scratch.data_ptr(),
                                      self.stream.cuda_stream))

    # ------------------------------------------------------------------ utils
    def _check(self, status: int) -> None:
        if status != 0:
            msg = self.lib.lbm_last_error(self.ctx)
            raise LBMError(status, msg.decode() if msg else "")

    def close(self) -> None:
        if getattr(self, "ctx", None):
            self.lib.lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -------------------------------------------------------------- the calls
    def init(self, seed: int, specs) -> None:
        if isinstance(specs, dict):
            specs = [specs] * len(self.lattices)
        arr = (_abi.lbm_init_spec * len(self.lattices))(*[_spec(s) for s in specs])
        self._check(self.lib.lbm_init(self.ctx, ctypes.c_uint64(seed), arr))

    def step(self, n: int = 1) -> None:
        self._check(self.lib.lbm_step(self.ctx, int(n)))

    @property
    def time(self) -> int:
        t = ctypes.c_int64()
        self._check(self.lib.lbm_get_time(self.ctx, ctypes.byref(t)))
        return t.value

    def moments(self, lattice: int = 0, out=None):
        """(rho, ux, uy) as FP32 CUDA tensors of shape (ny, nx)."""
        torch = self._torch
        L = self.lattices[lattice]
        if out is None:
            out = tuple(torch.empty((L.ny, L.nx), dtype=torch.float32, device=self.device) for _ in range(3))
        self._check(self.lib.lbm_moments(self.ctx, lattice, out[0].data_ptr(), out[1].data_ptr(),
                                         out[2].data_ptr()))
        self.stream.synchronize()
        return out

    def observables(self, lattice: int = 0) -> dict:
        o = _abi.lbm_obs()
        self._check(self.lib.lbm_observables(self.ctx, lattice, ctypes.byref(o)))
        return {k: getattr(o, k) for k, _ in _abi.lbm_obs._fields_}

    def observable_series(self, lattice: int = 0, cap: int = 1 << 20) -> list:
        buf = (_abi.lbm_obs * cap)()
        n = ctypes.c_int32()
        self._check(self.lib.lbm_observable_series(self.ctx, lattice, buf, cap, ctypes.byref(n)))
        return [{k: getattr(buf[i], k) for k, _ in _abi.lbm_obs._fields_} for i in range(n.value)]

    def get_state(self, lattice: int = 0, host: bool = False, out=None):
        """Populations as dense FP32 (Q, ny, nx); a (pinned) CPU tensor if host."""
        torch = self._torch
        L = self.lattices[lattice]
        if out is not None:
            if tuple(out.shape) != (L.q, L.ny, L.nx) or out.dtype != torch.float32 or not out.is_contiguous():
                raise ValueError(f"out must be a contiguous float32 ({L.q}, ny, nx) tensor")
            host = out.device.type == "cpu"
        elif host:
            out = torch.empty((L.q, L.ny, L.nx), dtype=torch.float32, pin_memory=True)
        else:
            out = torch.empty((L.q, L.ny, L.nx), dtype=torch.float32, device=self.device)
        self._check(self.lib.lbm_get_state(self.ctx, lattice, out.data_ptr(), 1 if host else 0))
        return out

    def set_state(self, f, lattice: int = 0) -> None:
        torch = self._torch
        L = self.lattices[lattice]
        f = torch.as_tensor(f)
        if tuple(f.shape) != (L.q, L.ny, L.nx):
            raise ValueError(f"state must have shape ({L.q}, {L.ny}, {L.nx})")
        f = f.to(torch.float32).contiguous()
        host = f.device.type == "cpu"
        if not host:
            self.stream.wait_stream(torch.cuda.current_stream(self.device))
        self._check(self.lib.lbm_set_state(self.ctx, lattice, f.data_ptr(), 1 if host else 0))

    def add_density(self, delta_rho_bar: float, lattice: int = -1) -> None:
        """Shift the mean density by delta (App. C.2), every lattice if -1."""
        self._check(self.lib.lbm_add_density(self.ctx, lattice, float(delta_rho_bar)))

    def set_params(self, params: dict, lattice: int = -1) -> None:
        """Replace the model parameters between steps (rho0 is kept)."""
        p = _params(params)
        self._check(self.lib.lbm_set_params(self.ctx, lattice, ctypes.byref(p)))

    def save(self, path: str) -> None:
        self._check(self.lib.lbm_save(self.ctx, str(path).encode()))

    def load(self, path: str) -> None:
        self._check(self.lib.lbm_load(self.ctx, str(path).encode()))

    def tune(self) -> None:
        self._check(self.lib.lbm_tune(self.ctx))

    def set_tuning(self, mode: int, vec: int = 1, rows: int = 32, warps: int = 4, stages: int = 0) -> None:
        """mode 0: automatic; mode 1: fixed shape (stages 0 = direct-load kernel,
        2..8 = shared-memory staged kernel with that many row buffers per warp)."""
        self._check(self.lib.lbm_set_tuning(self.ctx, mode, vec, rows, warps, stages))

    def get_tuning(self, lattice: int = 0) -> tuple:
        """(vec, rows, warps, stages) of the launch shape in use."""
        v, r, w, s = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self._check(self.lib.lbm_get_tuning(self.ctx, lattice, ctypes.byref(v), ctypes.byref(r), ctypes.byref(w),
                                            ctypes.byref(s)))
        return v.value, r.value, w.value, s.value

    def set_graphs(self, enabled: bool) -> None:
        self._check(self.lib.lbm_set_graphs(self.ctx, 1 if enabled else 0))

    def set_persistent(self, mode, l2_group_mib: int = 0) -> None:
        """Persistent launches of stretches of plain steps (groups on a direct
        kernel, either lattice): False/0 off, True/1 on, "auto"/2 chosen per
        group by the tuner; l2_group_mib MiB of populations per lattice group
        (0: one group)."""
        m = 2 if mode == "auto" else int(mode)
        self._check(self.lib.lbm_set_persistent(self.ctx, m, int(l2_group_mib)))

    def get_persistent(self, lattice: int = 0) -> bool:
        """Whether the lattice's launch group runs persistent launches now."""
        v = ctypes.c_int32()
        self._check(self.lib.lbm_get_persistent(self.ctx, lattice, ctypes.byref(v)))
        return bool(v.value)

    def last_launch_count(self) -> int:
        c = ctypes.c_int64()
        self._check(self.lib.lbm_last_launch_count(self.ctx, ctypes.byref(c)))
        return c.value

    def set_profiling(self, enabled: bool) -> None:
        self._check(self.lib.lbm_set_profiling(self.ctx, 1 if enabled else 0))

    def profile_read(self) -> dict:
        """Summed device ms of the fused step kernels and of the other kernels."""
        sm, om, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        self._check(self.lib.lbm_profile_read(self.ctx, ctypes.byref(sm), ctypes.byref(n), ctypes.byref(om)))
        return dict(step_ms=sm.value, step_launches=n.value, other_ms=om.value)

    def synchronize(self) -> None:
        self.stream.synchronize()
