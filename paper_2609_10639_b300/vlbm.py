"""Python binding of the VLBM step library (include/vlbm.h): argument marshalling only.

Every step of the method runs in the CUDA library libvlbm.so (built in-tree for sm_103a);
PyTorch supplies device memory and the stream.  There is no CPU fallback: if the library cannot
be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libvlbm.so")

OK, E_INVAL, E_NOMEM, E_CUDA, E_NONPHYSICAL, E_TIMEOUT, E_STATE, E_CHECKSUM, E_UNSUPPORTED = range(9)
BC = {"periodic": 0, "zerograd": 1, "inflow": 2}
PRECISION = {"fp64": 0, "fp32_store": 1}
ALGORITHM = {"auto": 0, "two_pass": 1, "lookahead": 2}
TILING = {"auto": 0, "tile": 1, "strip": 2}


class VLBMError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {_lib.vlbm_status_string(status).decode()} (status {status})")


class NonPhysicalState(VLBMError):
    pass


class _Grid(C.Structure):
    _fields_ = [("dim", C.c_int32), ("nx", C.c_int64), ("ny", C.c_int64), ("x0", C.c_double), ("x1", C.c_double),
                ("y0", C.c_double), ("y1", C.c_double), ("bc", C.c_int32 * 4)]


class _Eos(C.Structure):
    _fields_ = [("kind", C.c_int32), ("gamma", C.c_double), ("a", C.c_double), ("b", C.c_double), ("R", C.c_double),
                ("cv", C.c_double), ("cv1", C.c_double), ("cv2", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("cfl", C.c_double), ("beta_mode", C.c_int32), ("beta_const", C.c_double), ("beta_min", C.c_double),
                ("beta_max", C.c_double), ("c_sensor", C.c_double), ("ducros_eps", C.c_double),
                ("retarget_every", C.c_int32), ("precision", C.c_int32), ("algorithm", C.c_int32),
                ("tiling", C.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libvlbm.so not built ({LIB_PATH}); run `python -m paper_2609_10639_b300.build`")
    L = C.CDLL(LIB_PATH)
    V, P, D, I32, I64 = C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_int32, C.c_int64
    sig = {
        "vlbm_create": [C.POINTER(_Grid), C.POINTER(_Eos), C.POINTER(_Params), V, C.POINTER(V)],
        "vlbm_destroy": [V],
        "vlbm_init": [V, V],
        "vlbm_step": [V, I64, C.c_double, C.POINTER(I64)],
        "vlbm_get_W": [V, V],
        "vlbm_get_beta": [V, V],
        "vlbm_get_populations": [V, V],
        "vlbm_get_time": [V, D, C.POINTER(I64), D],
        "vlbm_get_dt_history": [V, V, V, I64, C.POINTER(I64)],
        "vlbm_set_dt_schedule": [V, V, I64],
        "vlbm_time_step_kernel": [V, I32, D],
        "vlbm_launches_per_step": [V, C.POINTER(I32)],
        "vlbm_set_profiling": [V, I32],
        "vlbm_adjoint": [V, V, I64, I32, V, V, D],
        "vlbm_adjoint_timing": [V, D, D],
        "vlbm_get_profile": [V, D, C.POINTER(I64)],
        "vlbm_get_totals": [V, D],
        "vlbm_save_state": [V, V, C.c_size_t, C.POINTER(C.c_size_t)],
        "vlbm_load_state": [V, V, C.c_size_t],
        "vlbm_measure_fp64_peak": [I32, D],
        "vlbm_set_inflow": [V, V],
        "vlbm_run_batch": [V, I64, C.POINTER(V), I64, C.c_double, C.POINTER(V), C.POINTER(I64)],
        "vlbm_set_adjoint_tape": [V, I64],
        "vlbm_adjoint_info": [V, D, C.POINTER(I64), C.POINTER(I64)],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.vlbm_status_string.argtypes = [C.c_int]
    L.vlbm_status_string.restype = C.c_char_p
    L.vlbm_version.argtypes = []
    L.vlbm_version.restype = C.c_char_p
    return L


_lib = _load()


def library():
    return _lib


def _check(status: int, what: str):
    if status == OK:
        return
    if status == E_NONPHYSICAL:
        raise NonPhysicalState(status, what)
    raise VLBMError(status, what)


def _eos_struct(e: dict) -> "_Eos":
    """vlbm_eos of an EOS description: ideal gas, van der Waals, or van der Waals with c_v(T)."""
    if e["kind"] == "ideal":
        return _Eos(0, e["gamma"], 0.0, 0.0, 0.0, 0.0, 0.0, 0.0)
    kind = 2 if e["kind"] == "vdw_cvt" else 1
    return _Eos(kind, 0.0, e["a"], e["b"], e["R"], e["cv"], e.get("cv1", 0.0), e.get("cv2", 0.0))


def _ptr(a) -> int:
    """Raw address of a contiguous float64 torch tensor (device or host) or numpy array."""
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "float64 C-contiguous array required"
        return a.ctypes.data
    assert a.dtype.itemsize == 8 and a.is_contiguous(), "contiguous float64 tensor required"
    return a.data_ptr()


def _ptr_n(a, n: int) -> int:
    """_ptr of an array that must hold exactly n values (the library writes or reads all of them)."""
    size = a.size if isinstance(a, np.ndarray) else a.numel()
    if size != n:
        raise ValueError(f"array of {size} values where {n} are required")
    return _ptr(a)


@dataclass
class Config:
    dim: int
    nx: int
    ny: int = 1
    extent: Sequence[float] = (0.0, 1.0, 0.0, 1.0)
    bc: Sequence[str] = ("zerograd",) * 4
    eos: dict = field(default_factory=lambda: {"kind": "ideal", "gamma": 1.4})
    cfl: float = 0.5
    beta_mode: str = "sensor"
    beta_const: float = 1.0
    beta_min: float = 0.75
    beta_max: float = 1.0
    c_sensor: float = 4.0
    ducros_eps: float = 1e-6
    retarget_every: int = 1
    precision: str = "fp64"
    algorithm: str = "auto"
    tiling: str = "auto"


class Solver:
    """A VLBM solver on the current CUDA device, bound to a torch CUDA stream."""

    def __init__(self, cfg: Config, stream=None):
        import torch

        self.torch = torch
        self.cfg = cfg
        self.dim = cfg.dim
        self.nx, self.ny = cfg.nx, (1 if cfg.dim == 1 else cfg.ny)
        self.nc, self.q = cfg.dim + 2, 2 * cfg.dim
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        g = _Grid(cfg.dim, cfg.nx, self.ny, *[float(v) for v in cfg.extent], (C.c_int32 * 4)(*[BC[b] for b in cfg.bc]))
        eo = _eos_struct(cfg.eos)
        p = _Params(cfg.cfl, 0 if cfg.beta_mode == "sensor" else 1, cfg.beta_const, cfg.beta_min, cfg.beta_max,
                    cfg.c_sensor, cfg.ducros_eps, cfg.retarget_every, PRECISION[cfg.precision], ALGORITHM[cfg.algorithm],
                    TILING[cfg.tiling])
        h = C.c_void_p()
        _check(_lib.vlbm_create(C.byref(g), C.byref(eo), C.byref(p), C.c_void_p(self.stream.cuda_stream), C.byref(h)),
               "vlbm_create")
        self._h = h

    @classmethod
    def for_problem(cls, prob, precision="fp64", algorithm="auto", stream=None, **over):
        kw = dict(dim=prob.dim, nx=prob.nx, ny=prob.ny, extent=prob.extent, bc=prob.bc, eos=prob.eos, cfl=prob.cfl,
                  beta_min=prob.beta_min, beta_max=prob.beta_max, c_sensor=prob.c_sensor, ducros_eps=prob.ducros_eps,
                  precision=precision, algorithm=algorithm)
        kw.update(over)
        s = cls(Config(**kw), stream=stream)
        if "inflow" in prob.bc:
            from . import workloads as wl

            s.set_inflow(wl.inflow_state(prob))
        return s

    def set_inflow(self, W_in) -> None:
        """State (D+2 conserved values) held by the ghost cells of the pinned-inflow x-lo side."""
        w = np.ascontiguousarray(np.asarray(W_in, dtype=np.float64).reshape(-1))
        _check(_lib.vlbm_set_inflow(self._h, C.c_void_p(w.ctypes.data)), "vlbm_set_inflow")

    def close(self):
        if getattr(self, "_h", None):
            _lib.vlbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.nc, self.ny, self.nx)

    def init(self, W0) -> None:
        if isinstance(W0, np.ndarray):
            W0 = np.ascontiguousarray(W0, dtype=np.float64).reshape(self.shape)
        _check(_lib.vlbm_init(self._h, C.c_void_p(_ptr_n(W0, self.nc * self.ny * self.nx))), "vlbm_init")
        self._keep = W0  # the copy is stream-ordered; keep the source alive until it ran

    def step(self, n_steps: int, t_end: float = 0.0) -> int:
        done = C.c_int64(0)
        _check(_lib.vlbm_step(self._h, int(n_steps), float(t_end), C.byref(done)), "vlbm_step")
        return done.value

    def W(self, out=None):
        if out is None:
            out = self.torch.empty(self.shape, dtype=self.torch.float64, device=self.device)
        _check(_lib.vlbm_get_W(self._h, C.c_void_p(_ptr_n(out, self.nc * self.ny * self.nx))), "vlbm_get_W")
        return out

    def run_batch(self, W0s, n_steps: int, t_end: float = 0.0, outs=None):
        """Independent runs init(W0s[k]) + step(n_steps, t_end) + W(outs[k]), host copies of one
        run overlapping the steps of the next (vlbm_run_batch).  Returns (outs, steps done)."""
        n = len(W0s)
        W0s = [np.ascontiguousarray(w, dtype=np.float64).reshape(self.shape) if isinstance(w, np.ndarray) else w
               for w in W0s]
        if outs is None:
            outs = [self.torch.empty(self.shape, dtype=self.torch.float64, device=self.device) for _ in range(n)]
        if len(outs) != n:
            raise ValueError("one output per input")
        m = self.nc * self.ny * self.nx
        ins = (C.c_void_p * n)(*[_ptr_n(w, m) for w in W0s])
        outp = (C.c_void_p * n)(*[_ptr_n(o, m) for o in outs])
        done = (C.c_int64 * n)()
        _check(_lib.vlbm_run_batch(self._h, n, ins, int(n_steps), float(t_end), outp, done), "vlbm_run_batch")
        return outs, list(done)

    def beta(self) -> np.ndarray:
        out = np.empty((self.ny, self.nx))
        _check(_lib.vlbm_get_beta(self._h, C.c_void_p(out.ctypes.data)), "vlbm_get_beta")
        return out

    def populations(self):
        out = self.torch.empty((self.q, self.nc, self.ny, self.nx), dtype=self.torch.float64, device=self.device)
        _check(_lib.vlbm_get_populations(self._h, C.c_void_p(out.data_ptr())), "vlbm_get_populations")
        return out

    def time(self):
        t, n, c = C.c_double(), C.c_int64(), C.c_double()
        _check(_lib.vlbm_get_time(self._h, C.byref(t), C.byref(n), C.byref(c)), "vlbm_get_time")
        return t.value, n.value, c.value

    def history(self):
        n = C.c_int64()
        _check(_lib.vlbm_get_dt_history(self._h, None, None, 0, C.byref(n)), "vlbm_get_dt_history")
        dt, c = np.empty(n.value), np.empty(n.value)
        _check(_lib.vlbm_get_dt_history(self._h, C.c_void_p(dt.ctypes.data), C.c_void_p(c.ctypes.data), n.value,
                                        C.byref(n)), "vlbm_get_dt_history")
        return dt, c

    def set_schedule(self, c) -> None:
        c = np.ascontiguousarray(c, dtype=np.float64)
        _check(_lib.vlbm_set_dt_schedule(self._h, C.c_void_p(c.ctypes.data) if len(c) else None, len(c)),
               "vlbm_set_dt_schedule")

    def time_step_kernel(self, reps: int = 10) -> float:
        ms = C.c_double()
        _check(_lib.vlbm_time_step_kernel(self._h, int(reps), C.byref(ms)), "vlbm_time_step_kernel")
        return ms.value

    def adjoint(self, W0, n_steps: int, checkpoint_every: int, dJ_dWT, dJ_dW0=None):
        """dJ/dW0 (CUDA tensor) and dJ/d(gamma, a, b, R, cv) (numpy) of an objective with gradient
        dJ_dWT at the final state of the run vlbm_init(W0) + n_steps steps (vlbm_adjoint)."""
        if dJ_dW0 is None:
            dJ_dW0 = self.torch.empty(self.shape, dtype=self.torch.float64, device=self.device)
        deos = np.zeros(5)
        _check(_lib.vlbm_adjoint(self._h, C.c_void_p(_ptr(W0)), int(n_steps), int(checkpoint_every),
                                 C.c_void_p(_ptr(dJ_dWT)), C.c_void_p(_ptr(dJ_dW0)),
                                 deos.ctypes.data_as(C.POINTER(C.c_double))), "vlbm_adjoint")
        return dJ_dW0, deos

    def adjoint_timing(self):
        """Device ms of the reverse pass of the last adjoint call, and of its segment
        recomputations alone."""
        ms, rc = C.c_double(), C.c_double()
        _check(_lib.vlbm_adjoint_timing(self._h, C.byref(ms), C.byref(rc)), "vlbm_adjoint_timing")
        return ms.value, rc.value

    def set_adjoint_tape(self, max_bytes: int) -> None:
        """Adjoint tape limit in bytes (< 0: 3/4 of the free device memory; 0: off)."""
        _check(_lib.vlbm_set_adjoint_tape(self._h, int(max_bytes)), "vlbm_set_adjoint_tape")

    def adjoint_info(self):
        """(forward-pass ms, taped steps, tape bytes) of the last adjoint call."""
        ms, n, b = C.c_double(), C.c_int64(), C.c_int64()
        _check(_lib.vlbm_adjoint_info(self._h, C.byref(ms), C.byref(n), C.byref(b)), "vlbm_adjoint_info")
        return ms.value, n.value, b.value

    def set_profiling(self, on: bool) -> None:
        _check(_lib.vlbm_set_profiling(self._h, 1 if on else 0), "vlbm_set_profiling")

    def profile(self):
        """(summed device ms of the bracketed step-kernel launches, number of launches)."""
        ms, n = C.c_double(), C.c_int64()
        _check(_lib.vlbm_get_profile(self._h, C.byref(ms), C.byref(n)), "vlbm_get_profile")
        return ms.value, n.value

    def totals(self) -> np.ndarray:
        """Compensated FP64 domain totals sum_x W_k of the current state (vlbm_get_totals)."""
        out = np.zeros(self.nc)
        _check(_lib.vlbm_get_totals(self._h, out.ctypes.data_as(C.POINTER(C.c_double))), "vlbm_get_totals")
        return out

    def save_state(self) -> bytes:
        """The complete state of the run as a checksummed byte string (vlbm_save_state)."""
        n = C.c_size_t()
        _check(_lib.vlbm_save_state(self._h, None, 0, C.byref(n)), "vlbm_save_state")
        buf = C.create_string_buffer(n.value)
        _check(_lib.vlbm_save_state(self._h, buf, n.value, C.byref(n)), "vlbm_save_state")
        return buf.raw

    def load_state(self, state: bytes) -> None:
        """Restores a state written by save_state on a solver of the same configuration."""
        buf = C.create_string_buffer(bytes(state), len(state))
        _check(_lib.vlbm_load_state(self._h, buf, len(state)), "vlbm_load_state")

    def launches_per_step(self) -> int:
        n = C.c_int32()
        _check(_lib.vlbm_launches_per_step(self._h, C.byref(n)), "vlbm_launches_per_step")
        return n.value


def _config_structs(cfg: Config):
    """(_Grid, _Eos, _Params) of a Config, for the handle-free entry point."""
    ny = 1 if cfg.dim == 1 else cfg.ny
    g = _Grid(cfg.dim, cfg.nx, ny, *[float(v) for v in cfg.extent], (C.c_int32 * 4)(*[BC[b] for b in cfg.bc]))
    e = cfg.eos
    eo = _eos_struct(e)
    p = _Params(cfg.cfl, 0 if cfg.beta_mode == "sensor" else 1, cfg.beta_const, cfg.beta_min, cfg.beta_max,
                cfg.c_sensor, cfg.ducros_eps, cfg.retarget_every, PRECISION[cfg.precision], ALGORITHM[cfg.algorithm],
                    TILING[cfg.tiling])
    return g, eo, p


_lib.vlbm_beta_noalloc.argtypes = [C.POINTER(_Grid), C.POINTER(_Eos), C.POINTER(_Params), C.c_void_p, C.c_int32,
                                   C.c_void_p, C.c_void_p]
_lib.vlbm_beta_noalloc.restype = C.c_int


def beta_noalloc(cfg: Config, f, out, in_place: bool = True, stream=None) -> None:
    """beta(x) of caller-owned FP64 populations `f` (CUDA tensor [2D][D+2][ny][nx]) into the
    caller-owned CUDA tensor `out` ([ny][nx]) without any device allocation (for callers that
    cannot allocate; see vlbm_beta_noalloc in include/vlbm.h).  Asynchronous on `stream`."""
    import torch

    g, eo, p = _config_structs(cfg)
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(_lib.vlbm_beta_noalloc(C.byref(g), C.byref(eo), C.byref(p), C.c_void_p(_ptr(f)), 1 if in_place else 0,
                                  C.c_void_p(_ptr(out)), C.c_void_p(s.cuda_stream)), "vlbm_beta_noalloc")


def measure_fp64_peak(reps: int = 5) -> float:
    """Measured FP64 throughput of the current GPU in TFLOP/s (vlbm_measure_fp64_peak)."""
    out = C.c_double(0.0)
    _check(_lib.vlbm_measure_fp64_peak(int(reps), C.byref(out)), "vlbm_measure_fp64_peak")
    return out.value
