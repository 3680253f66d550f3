"""ORACLE: test infrastructure only (ctypes wrapper around vlbm_oracle.cpp).

Only the tests, the package smoke check and the CPU-baseline leg of the benchmark may import
this module.  It builds the plain FP64 C++ oracle on first use (g++ -O2 -ffp-contract=off
-fopenmp) and exposes it with numpy arrays.  See vlbm_oracle.cpp for what each call computes
and which passage of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "vlbm_oracle.cpp")
SRCS = [SRC, os.path.join(HERE, "muscl_reference.cpp")]
LIB = os.path.join(HERE, "liboracle_vlbm.so")
_lock = threading.Lock()
_lib = None

BC_CODE = {"periodic": 0, "zerograd": 1, "inflow": 2}


def build(force: bool = False) -> str:
    """Compile the oracle shared library next to its source (no fused multiply-add)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(s) for s in SRCS):
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", LIB, *SRCS]
        subprocess.run(cmd, check=True)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            P, D, I, Lg = C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_long
            sig = {
                "orc_create": (P, [I, Lg, Lg, C.c_double, C.POINTER(C.c_int), D, D]),
                "orc_destroy": (None, [P]),
                "orc_set_threads": (None, [P, I]),
                "orc_max_threads": (I, []),
                "orc_init": (I, [P, D]),
                "orc_step": (I, [P, Lg, C.c_double, C.POINTER(C.c_long)]),
                "orc_get_W": (None, [P, D]),
                "orc_get_f": (None, [P, D]),
                "orc_set_state": (None, [P, D, C.c_double, C.c_double, Lg]),
                "orc_get_beta": (None, [P, D]),
                "orc_eval_beta": (I, [P, D]),
                "orc_eval_sensor_fields": (I, [P, D, D, D, D, D]),
                "orc_get_time": (None, [P, D, C.POINTER(C.c_long), D]),
                "orc_get_hist": (Lg, [P, D, D, Lg]),
                "orc_set_schedule": (None, [P, D, Lg]),
                "orc_set_inflow": (I, [P, D]),
                "orc_dual_set_inflow": (I, [P, D]),
                "orc_eos_eval": (None, [D, C.c_double, C.c_double, D, D]),
                "orc_fundamental_derivative": (C.c_double, [D, C.c_double, C.c_double]),
                "orc_flux": (I, [I, D, D, D]),
                "orc_feq": (I, [I, D, C.c_double, D, D]),
                "orc_reproject": (None, [I, C.c_double, C.c_double, D]),
                "orc_dual_create": (P, [I, Lg, Lg, C.c_double, C.POINTER(C.c_int), D, D, D]),
                "orc_dual_destroy": (None, [P]),
                "orc_dual_set_threads": (None, [P, I]),
                "orc_dual_set_schedule": (None, [P, D, Lg]),
                "orc_dual_init": (I, [P, D, D]),
                "orc_dual_step": (I, [P, Lg, C.POINTER(C.c_long)]),
                "orc_dual_get_W": (None, [P, D, D]),
                "orc_muscl_1d": (I, [D, I, C.c_double, I, C.c_double, C.c_double, D, C.POINTER(C.c_long)]),
                "orc_muscl_2d": (I, [D, I, I, C.c_double, C.c_double, C.c_double, D, C.POINTER(C.c_long)]),
                "orc_muscl_2d_bc": (I, [D, I, I, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_int), D, D,
                                        C.POINTER(C.c_long)]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def eos6(eos: dict) -> np.ndarray:
    """EOS parameters as the C entry points read them: kind, gamma, a, b, R, cv, cv1, cv2."""
    if eos["kind"] == "ideal":
        return np.array([0.0, eos["gamma"], 0.0, 0.0, 0.0, 0.0, 0.0, 0.0])
    kind = 2.0 if eos["kind"] == "vdw_cvt" else 1.0
    return np.array([kind, 1.0 + eos["R"] / eos["cv"], eos["a"], eos["b"], eos["R"], eos["cv"], eos.get("cv1", 0.0),
                     eos.get("cv2", 0.0)])


def prm8(cfl=0.5, beta_mode="sensor", beta_const=1.0, beta_min=0.75, beta_max=1.0, c_sensor=4.0, ducros_eps=1e-6,
         retarget_every=1) -> np.ndarray:
    return np.array([cfl, 0.0 if beta_mode == "sensor" else 1.0, beta_const, beta_min, beta_max, c_sensor, ducros_eps,
                     float(retarget_every)])


class OracleSolver:
    """The oracle's solver: populations f[i][k][y][x] in FP64, advanced by the paper's cycle."""

    def __init__(self, dim, nx, ny, dx, bc, eos: dict, threads: int | None = None, **params):
        self.L = lib()
        self.dim, self.nx, self.ny = dim, nx, (1 if dim == 1 else ny)
        self.nc, self.q = dim + 2, 2 * dim
        self.eos = eos
        bc4 = (C.c_int * 4)(*[BC_CODE[b] for b in bc])
        self._e6 = eos6(eos)
        self._p8 = prm8(**params)
        self.h = self.L.orc_create(dim, nx, self.ny, dx, bc4, _dp(self._e6), _dp(self._p8))
        n = threads if threads is not None else int(os.environ.get("ORACLE_THREADS", "0")) or self.L.orc_max_threads()
        self.threads = n
        self.L.orc_set_threads(self.h, n)

    @classmethod
    def for_problem(cls, p, threads=None, **over):
        params = dict(cfl=p.cfl, beta_min=p.beta_min, beta_max=p.beta_max, c_sensor=p.c_sensor,
                      ducros_eps=p.ducros_eps)
        params.update(over)
        s = cls(p.dim, p.nx, p.ny, p.dx, p.bc, p.eos, threads=threads, **params)
        if "inflow" in p.bc:
            from paper_2609_10639_b300 import workloads as wl

            s.set_inflow(wl.inflow_state(p))
        return s

    def set_inflow(self, W_in) -> None:
        """State (D+2 conserved values) held by the ghost cells of the pinned-inflow x-lo side."""
        w = np.ascontiguousarray(np.asarray(W_in, dtype=np.float64).reshape(-1))
        if self.L.orc_set_inflow(self.h, _dp(w)):
            raise ValueError("oracle set_inflow: non-physical state")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.orc_destroy(h)
            self.h = None

    @property
    def shape(self):
        return (self.nc, self.ny, self.nx)

    def init(self, W0: np.ndarray) -> None:
        W0 = np.ascontiguousarray(W0, dtype=np.float64).reshape(self.shape)
        st = self.L.orc_init(self.h, _dp(W0))
        if st:
            raise ValueError(f"oracle init: non-physical state (status {st})")

    def step(self, n_steps: int, t_end: float = 0.0) -> int:
        done = C.c_long(0)
        st = self.L.orc_step(self.h, n_steps, t_end, C.byref(done))
        if st:
            raise ValueError(f"oracle step: non-physical state (status {st}) after {done.value} steps")
        return done.value

    def W(self) -> np.ndarray:
        out = np.empty(self.shape)
        self.L.orc_get_W(self.h, _dp(out))
        return out

    def f(self) -> np.ndarray:
        out = np.empty((self.q, self.nc, self.ny, self.nx))
        self.L.orc_get_f(self.h, _dp(out))
        return out

    def set_state(self, f: np.ndarray, c_prev: float, t: float = 0.0, n: int = 0) -> None:
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.q, self.nc, self.ny, self.nx)
        self.L.orc_set_state(self.h, _dp(f), c_prev, t, n)

    def beta(self) -> np.ndarray:
        """beta(x) used by the last step."""
        out = np.empty((self.ny, self.nx))
        self.L.orc_get_beta(self.h, _dp(out))
        return out

    def eval_beta(self) -> np.ndarray:
        """beta(x) of the current state (no step taken)."""
        out = np.empty((self.ny, self.nx))
        st = self.L.orc_eval_beta(self.h, _dp(out))
        if st:
            raise ValueError("oracle eval_beta: non-physical state")
        return out

    def sensor_fields(self) -> dict:
        """The shock sensor's fields of the current state (no step taken): s and theta before
        the box filter, s_bar and theta_bar after it, and beta (theta = 0 in 1D)."""
        out = {k: np.empty((self.ny, self.nx)) for k in ("s", "theta", "s_bar", "theta_bar", "beta")}
        st = self.L.orc_eval_sensor_fields(self.h, *[_dp(out[k]) for k in ("s", "theta", "s_bar", "theta_bar", "beta")])
        if st:
            raise ValueError("oracle sensor_fields: non-physical state")
        return out

    def time(self):
        t = C.c_double()
        n = C.c_long()
        c = C.c_double()
        self.L.orc_get_time(self.h, C.byref(t), C.byref(n), C.byref(c))
        return t.value, n.value, c.value

    def history(self):
        n = self.L.orc_get_hist(self.h, None, None, 0)
        dt, c = np.empty(n), np.empty(n)
        self.L.orc_get_hist(self.h, _dp(dt), _dp(c), n)
        return dt, c

    def set_schedule(self, c: np.ndarray) -> None:
        c = np.ascontiguousarray(c, dtype=np.float64)
        self.L.orc_set_schedule(self.h, _dp(c), len(c))


class DualOracleSolver:
    """The same solver in first-order dual numbers along one direction (dW0, deos)."""

    def __init__(self, dim, nx, ny, dx, bc, eos: dict, deos: dict | None = None, threads: int | None = None, **params):
        self.L = lib()
        self.dim, self.nx, self.ny = dim, nx, (1 if dim == 1 else ny)
        self.nc = dim + 2
        bc4 = (C.c_int * 4)(*[BC_CODE[b] for b in bc])
        self._e6 = eos6(eos)
        self._de6 = np.zeros(8)
        for j, key in enumerate(["kind", "gamma", "a", "b", "R", "cv", "cv1", "cv2"]):
            if deos and key in deos:
                self._de6[j] = deos[key]
        self._p8 = prm8(**params)
        self.h = self.L.orc_dual_create(dim, nx, self.ny, dx, bc4, _dp(self._e6), _dp(self._de6), _dp(self._p8))
        n = threads if threads is not None else self.L.orc_max_threads()
        self.L.orc_dual_set_threads(self.h, n)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.orc_dual_destroy(h)
            self.h = None

    def set_schedule(self, c: np.ndarray) -> None:
        c = np.ascontiguousarray(c, dtype=np.float64)
        self.L.orc_dual_set_schedule(self.h, _dp(c), len(c))

    def set_inflow(self, W_in) -> None:
        w = np.ascontiguousarray(np.asarray(W_in, dtype=np.float64).reshape(-1))
        if self.L.orc_dual_set_inflow(self.h, _dp(w)):
            raise ValueError("dual oracle set_inflow: non-physical state")

    def init(self, W0: np.ndarray, dW0: np.ndarray | None) -> None:
        shape = (self.nc, self.ny, self.nx)
        W0 = np.ascontiguousarray(W0, dtype=np.float64).reshape(shape)
        d = np.zeros(shape) if dW0 is None else np.ascontiguousarray(dW0, dtype=np.float64).reshape(shape)
        if self.L.orc_dual_init(self.h, _dp(W0), _dp(d)):
            raise ValueError("dual oracle init: non-physical state")

    def step(self, n_steps: int) -> int:
        done = C.c_long(0)
        if self.L.orc_dual_step(self.h, n_steps, C.byref(done)):
            raise ValueError(f"dual oracle step failed after {done.value} steps")
        return done.value

    def W(self):
        shape = (self.nc, self.ny, self.nx)
        W, dW = np.empty(shape), np.empty(shape)
        self.L.orc_dual_get_W(self.h, _dp(W), _dp(dW))
        return W, dW


# --- point functions ---
def eos_eval(eos: dict, rho: float, e: float):
    P, cs2 = C.c_double(), C.c_double()
    e6 = eos6(eos)
    lib().orc_eos_eval(_dp(e6), rho, e, C.byref(P), C.byref(cs2))
    return P.value, cs2.value


def fundamental_derivative(eos: dict, rho: float, e: float) -> float:
    e6 = eos6(eos)
    return lib().orc_fundamental_derivative(_dp(e6), rho, e)


def flux(dim: int, eos: dict, W) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.float64)
    out = np.empty(dim * (dim + 2))
    e6 = eos6(eos)
    if lib().orc_flux(dim, _dp(e6), _dp(W), _dp(out)):
        raise ValueError("non-physical state")
    return out.reshape(dim, dim + 2)


def feq(dim: int, eos: dict, c: float, W) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.float64)
    out = np.empty(2 * dim * (dim + 2))
    e6 = eos6(eos)
    if lib().orc_feq(dim, _dp(e6), c, _dp(W), _dp(out)):
        raise ValueError("non-physical state")
    return out.reshape(2 * dim, dim + 2)


def reproject(dim: int, c_old: float, c_new: float, f) -> np.ndarray:
    f = np.array(f, dtype=np.float64).reshape(-1).copy()
    lib().orc_reproject(dim, c_old, c_new, _dp(f))
    return f.reshape(2 * dim, dim + 2)


def muscl_1d(eos: dict, W0, dx: float, bc: str, t_end: float, cfl: float = 0.4):
    """The independent reference method (muscl_reference.cpp): MUSCL-minmod in primitive
    variables, Rusanov flux, Heun RK2, from W0 (3 x n conserved) at t = 0 to t_end.  Returns
    (W(t_end), steps)."""
    W = np.ascontiguousarray(np.asarray(W0, dtype=np.float64).reshape(3, -1)).copy()
    steps = C.c_long(0)
    e6 = eos6(eos)
    st = lib().orc_muscl_1d(_dp(e6), W.shape[1], dx, BC_CODE[bc], cfl, t_end, _dp(W), C.byref(steps))
    if st:
        raise ValueError(f"MUSCL reference: non-physical state after {steps.value} steps")
    return W, steps.value


def muscl_2d(eos: dict, W0, dx: float, t_end: float, cfl: float = 0.4, bc=("zerograd",) * 4, W_in=None):
    """The reference method in 2D (muscl_reference.cpp): unsplit, from W0 (4 x ny x nx conserved)
    at t = 0 to t_end, with per-side boundaries (periodic, zero-gradient, or "inflow": ghost cells
    holding the conserved state W_in).  Returns (W(t_end), steps)."""
    W = np.ascontiguousarray(np.asarray(W0, dtype=np.float64)).copy()
    _, ny, nx = W.shape
    steps = C.c_long(0)
    e6 = eos6(eos)
    bc4 = (C.c_int * 4)(*[BC_CODE[b] for b in bc])
    win = None if W_in is None else np.ascontiguousarray(np.asarray(W_in, dtype=np.float64).reshape(-1))
    st = lib().orc_muscl_2d_bc(_dp(e6), nx, ny, dx, cfl, t_end, bc4, None if win is None else _dp(win), _dp(W),
                               C.byref(steps))
    if st:
        raise ValueError(f"MUSCL reference (2D): non-physical state after {steps.value} steps")
    return W, steps.value
