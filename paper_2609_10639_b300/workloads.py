"""Seeded synthetic inputs for the VLBM step: initial fields W0, objective weights, directions.

This module only builds inputs.  It contains none of the time step's arithmetic (no
equilibrium, flux, sensor, relaxation or streaming); the one piece of thermodynamics here is the
conversion of a primitive state (rho, u, v, P) into the conserved vector
W = (rho, rho u, rho v, rho E) of Sec. II A (Eqs. 1-2), which is how every initial condition of
the paper is stated.

Random numbers come from splitmix64 (Steele, Lea & Flood 2014) mapped to 53-bit doubles, so the
same seed gives the same fields on every platform.  Field arrays are float64, shaped
(D+2, ny, nx) with x fastest (1D problems have ny = 1).  Cell centres are x_j = x0 + (j + 1/2) dx.
"""
from __future__ import annotations

import dataclasses
import json
import math
import os
from typing import Callable, Optional, Sequence

import numpy as np

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64 stream: state += 0x9E3779B97F4A7C15, then the published mix of the state."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        """Uniform double in [lo, hi) from the top 53 bits."""
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def integer(self, lo: int, hi: int) -> int:
        """Integer in [lo, hi] (inclusive)."""
        return lo + min(int(self.uniform() * (hi - lo + 1)), hi - lo)


# ------------------------------------------------------------------------------------------
# Problem descriptions (plain data).
# ------------------------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Problem:
    name: str
    dim: int
    nx: int
    ny: int
    extent: tuple  # (x0, x1, y0, y1)
    bc: tuple  # (x-lo, x-hi, y-lo, y-hi): "periodic" | "zerograd" | "inflow" (x-lo only, pinned state)
    eos: dict  # {"kind": "ideal", "gamma": g} | {"kind": "vdw", "a", "b", "R", "cv"}
    cfl: float
    t_end: float  # 0: run a fixed number of steps
    n_steps: int  # steps of a full run (0: run to t_end)
    beta_min: float = 0.75
    beta_max: float = 1.0
    c_sensor: float = 4.0
    ducros_eps: float = 1e-6

    @property
    def dx(self) -> float:
        return (self.extent[1] - self.extent[0]) / self.nx

    @property
    def ncells(self) -> int:
        return self.nx * self.ny

    def resized(self, nx: int, ny: Optional[int] = None) -> "Problem":
        return dataclasses.replace(self, nx=nx, ny=(1 if self.dim == 1 else (ny if ny is not None else nx)))


IDEAL14 = {"kind": "ideal", "gamma": 1.4}
# Reduced van der Waals units (rho_c = P_c = T_c = 1): a = 3, b = 1/3, R = 8/3, cv = 50 R.
VDW_REDUCED = {"kind": "vdw", "a": 3.0, "b": 1.0 / 3.0, "R": 8.0 / 3.0, "cv": 50.0 * 8.0 / 3.0}
# The same gas with a temperature-dependent heat capacity c_v(T) = R (40 + 8 T + 2 T^2) (50 R at the
# critical temperature T = 1): a non-polytropic closure whose e -> T inversion needs Newton's method.
VDW_CVT_REDUCED = {"kind": "vdw_cvt", "a": 3.0, "b": 1.0 / 3.0, "R": 8.0 / 3.0, "cv": 40.0 * 8.0 / 3.0,
                   "cv1": 8.0 * 8.0 / 3.0, "cv2": 2.0 * 8.0 / 3.0}

ZG = ("zerograd",) * 4
PER = ("periodic",) * 4

SOD_1D = Problem("sod_1d_1000", 1, 1000, 1, (0.0, 1.0, 0.0, 0.0), ZG, IDEAL14, 0.5, 0.2, 0)
QUADRANTS_2D = Problem("quadrants_2d_4096", 2, 4096, 4096, (0.0, 1.0, 0.0, 1.0), ZG, IDEAL14, 0.5, 0.25, 0)
BZT_2D = Problem("bzt_interface_2d_2048", 2, 2048, 2048, (0.0, 1.0, 0.0, 1.0), ZG, VDW_REDUCED, 0.5, 0.2, 0)
# The BZT interface input with the non-polytropic gas (the same seeded states and perturbation).
BZT_CVT_2D = Problem("bzt_interface_cvt_2d_2048", 2, 2048, 2048, (0.0, 1.0, 0.0, 1.0), ZG, VDW_CVT_REDUCED, 0.5, 0.2, 0)
VORTEX_SCALE_2D = Problem("vortex_acoustic_2d_8192", 2, 8192, 8192, (0.0, 10.0, 0.0, 10.0), PER, IDEAL14, 0.5, 0.0, 2000)
VORTEX_ADJOINT_2D = Problem("vortex_adjoint_2d_1024", 2, 1024, 1024, (0.0, 10.0, 0.0, 10.0), PER, IDEAL14, 0.5, 0.0, 1000)

# One-dimensional accuracy benchmarks of Secs. IV B-IV D, run against the independent reference
# solver: the strong shock tube (Sec. IV C, N = 2000, CFL 0.8) and the Shu-Osher problem
# (Sec. IV B, x in [-5, 5], t = 1.9, CFL 0.8); the van der Waals shock tubes are argrow_1d().
STRONG_SHOCK_1D = Problem("strong_shock_1d_2000", 1, 2000, 1, (0.0, 1.0, 0.0, 0.0), ZG, IDEAL14, 0.8, 0.012, 0)
SHU_OSHER_1D = Problem("shu_osher_1d_2000", 1, 2000, 1, (-5.0, 5.0, 0.0, 0.0), ZG, IDEAL14, 0.8, 1.9, 0)

# Gresho vortex (Sec. IV A): periodic [0,1]^2, gamma = 5/3, the exact steady solution run to
# t = 0.5 (CFL 0.5: the paper does not state it for this case).
GRESHO_2D = Problem("gresho_2d_128", 2, 128, 128, (0.0, 1.0, 0.0, 1.0), PER, {"kind": "ideal", "gamma": 5.0 / 3.0}, 0.5,
                    0.5, 0)

# Shock-vortex interaction (Sec. IV H): [0,16] x [0,6], stationary normal shock at x = 6 (M_s = 1.2),
# isentropic vortex (beta_v = 2, R_c = 1) at (2, 3) in the upstream flow; left side pinned to the
# upstream state, right side zero-gradient (outflow), y periodic.  CFL 0.5 (not stated for this case).
INFLOW_BC = ("inflow", "zerograd", "periodic", "periodic")
BZT_SV_EOS = {"kind": "vdw", "a": 1.0, "b": 0.3, "R": 1.0, "cv": 50.0}
SHOCK_VORTEX_IDEAL = Problem("shock_vortex_ideal_800x300", 2, 800, 300, (0.0, 16.0, 0.0, 6.0), INFLOW_BC, IDEAL14, 0.5,
                             7.0, 0)
SHOCK_VORTEX_BZT = Problem("shock_vortex_bzt_1200x450", 2, 1200, 450, (0.0, 16.0, 0.0, 6.0), INFLOW_BC, BZT_SV_EOS,
                           0.5, 15.0, 0)

PROBLEMS = {p.name: p for p in (SOD_1D, QUADRANTS_2D, BZT_2D, BZT_CVT_2D, VORTEX_SCALE_2D, VORTEX_ADJOINT_2D, STRONG_SHOCK_1D,
                                SHU_OSHER_1D, GRESHO_2D, SHOCK_VORTEX_IDEAL, SHOCK_VORTEX_BZT)}


def cell_centres(p: Problem):
    x0, x1, y0, y1 = p.extent
    dx = p.dx
    x = x0 + (np.arange(p.nx) + 0.5) * dx
    if p.dim == 1:
        return x[None, :], np.zeros((1, p.nx))
    y = y0 + (np.arange(p.ny) + 0.5) * dx
    X, Y = np.meshgrid(x, y, indexing="xy")
    return X, Y


# ------------------------------------------------------------------------------------------
# Primitive -> conserved (Sec. II A, Eqs. 1-2) with the internal energy of the closure
# (Eq. 15 ideal gas; Eqs. 16-17 van der Waals solved for T, then e = cv T - a rho).
# ------------------------------------------------------------------------------------------
def internal_energy(eos: dict, rho, P):
    """e of (rho, P): ideal gas (Eq. 15); van der Waals T from Eq. (16), then e = cv T - a rho
    (Eq. 17), or, for the temperature-dependent heat capacity c_v(T) = cv + cv1 T + cv2 T^2
    ("vdw_cvt"), e = cv T + cv1 T^2/2 + cv2 T^3/3 - a rho."""
    if eos["kind"] == "ideal":
        return P / ((eos["gamma"] - 1.0) * rho)
    a, b, R, cv = eos["a"], eos["b"], eos["R"], eos["cv"]
    T = (P + a * rho * rho) * (1.0 - b * rho) / (R * rho)
    if eos["kind"] == "vdw_cvt":
        return cv * T + eos["cv1"] * T * T / 2.0 + eos["cv2"] * T * T * T / 3.0 - a * rho
    return cv * T - a * rho


def vdw_pressure_at_T(eos: dict, rho, T):
    a, b, R = eos["a"], eos["b"], eos["R"]
    return R * rho * T / (1.0 - b * rho) - a * rho * rho


def vdw_temperature(eos: dict, rho, P):
    a, b, R = eos["a"], eos["b"], eos["R"]
    return (P + a * rho * rho) * (1.0 - b * rho) / (R * rho)


def conserved(eos: dict, rho, vel: Sequence, P) -> np.ndarray:
    rho = np.asarray(rho, dtype=np.float64)
    vel = [np.asarray(v, dtype=np.float64) for v in vel]
    e = internal_energy(eos, rho, np.asarray(P, dtype=np.float64))
    ke = 0.5 * sum(v * v for v in vel)
    comps = [rho] + [rho * v for v in vel] + [rho * (e + ke)]
    return np.ascontiguousarray(np.stack([np.broadcast_to(c, rho.shape) for c in comps]).astype(np.float64))


# ------------------------------------------------------------------------------------------
# Initial conditions
# ------------------------------------------------------------------------------------------
def sod_1d(p: Problem = SOD_1D, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1), x_interface=0.5) -> np.ndarray:
    """Two-state 1D Riemann problem: (rho, u, P) left / right of x_interface."""
    X, _ = cell_centres(p)
    L = X < x_interface
    rho = np.where(L, left[0], right[0])
    u = np.where(L, left[1], right[1])
    P = np.where(L, left[2], right[2])
    return conserved(p.eos, rho, [u], P)


_QUAD_SEED_FILE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                               "quadrant_seed.json")


def quadrant_seed() -> int:
    """Seed of the four-quadrant input: the first seed (from 2 up) whose states the oracle advances
    to t = 0.25 on a 512 x 512 copy without leaving the physical states (stored beside the
    fixture script that chose it)."""
    with open(_QUAD_SEED_FILE) as fh:
        return int(json.load(fh)["seed"])


def quadrant_states(seed: Optional[int] = None):
    """Four (rho, u, v, P) states in NE, NW, SW, SE order; per state rho~U[0.1,2], u,v~U[-1,1],
    P~U[0.05,2], drawn in that order."""
    g = SplitMix64(quadrant_seed() if seed is None else seed)
    out = []
    for _ in range(4):
        rho = g.uniform(0.1, 2.0)
        u = g.uniform(-1.0, 1.0)
        v = g.uniform(-1.0, 1.0)
        P = g.uniform(0.05, 2.0)
        out.append((rho, u, v, P))
    return out


def quadrants_2d(p: Problem = QUADRANTS_2D, seed: Optional[int] = None, states=None) -> np.ndarray:
    """Four-quadrant 2D Riemann problem with the discontinuities on x = 0.5 and y = 0.5."""
    st = states if states is not None else quadrant_states(seed)
    X, Y = cell_centres(p)
    xm = 0.5 * (p.extent[0] + p.extent[1])
    ym = 0.5 * (p.extent[2] + p.extent[3])
    E, N = X >= xm, Y >= ym
    masks = [E & N, ~E & N, ~E & ~N, E & ~N]  # NE, NW, SW, SE
    fields = [np.zeros(X.shape) for _ in range(4)]
    for m, s in zip(masks, st):
        for j in range(4):
            fields[j][m] = s[j]
    rho, u, v, P = fields
    return conserved(p.eos, rho, [u, v], P)


def draw_bzt_candidates(seed: int, count: int):
    """Candidate left/right (rho, P) pairs in [0.4, 0.95] x [0.8, 1.15], drawn rho then P."""
    g = SplitMix64(seed)
    return [(g.uniform(0.4, 0.95), g.uniform(0.8, 1.15)) for _ in range(count)]


_BZT_STATES_FILE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                                "bzt_states_seed3.json")


def bzt_states(seed: int = 3, accept: Optional[Callable[[float, float], bool]] = None,
               pair_ok: Optional[Callable[[tuple, tuple], bool]] = None):
    """Left and right (rho, P) states of the BZT interface problem.  Candidates come from the
    seed's stream; a candidate state is kept where `accept` holds (c_s^2 > 0 and fundamental
    derivative Gamma < 0); consecutive kept states form (left, right) pairs, and the first pair for
    which `pair_ok` holds (the flow it starts stays hyperbolic, Eq. 14) is returned.  Without
    predicates, the pair stored for seed 3 (written by the fixture script beside the file, from the
    oracle) is returned."""
    if accept is None:
        with open(_BZT_STATES_FILE) as fh:
            d = json.load(fh)
        if d["seed"] != seed:
            raise ValueError(f"stored BZT states are for seed {d['seed']}, not {seed}")
        return [tuple(d["left"]), tuple(d["right"])]
    kept = []
    for rho, P in draw_bzt_candidates(seed, 20000):
        if not accept(rho, P):
            continue
        kept.append((rho, P))
        if len(kept) == 2:
            if pair_ok is None or pair_ok(kept[0], kept[1]):
                return kept
            kept = []
    raise RuntimeError("no accepted BZT state pair in 20000 draws")


def bzt_interface_2d(p: Problem = BZT_2D, seed: int = 3, states=None, amp: float = 1e-3, modes: int = 16) -> np.ndarray:
    """Planar interface at x = 0.5 between two van der Waals states at rest, with the density
    multiplied by 1 + amp * mean_m cos(2 pi (n_x x + n_y y) + phi_m) at fixed temperature;
    n_x, n_y ~ integers in [1, 8], phi ~ U[0, 2 pi), drawn from seed + 1000."""
    (rl, Pl), (rr, Pr) = states if states is not None else bzt_states(seed)
    X, Y = cell_centres(p)
    L = X < 0.5 * (p.extent[0] + p.extent[1])
    rho0 = np.where(L, rl, rr)
    T = np.where(L, vdw_temperature(p.eos, rl, Pl), vdw_temperature(p.eos, rr, Pr))
    g = SplitMix64(seed + 1000)
    pert = np.zeros(X.shape)
    for _ in range(modes):
        nx_, ny_ = g.integer(1, 8), g.integer(1, 8)
        phi = g.uniform(0.0, 2.0 * math.pi)
        pert += np.cos(2.0 * math.pi * (nx_ * X + ny_ * Y) + phi)
    rho = rho0 * (1.0 + amp * pert / modes)
    P = vdw_pressure_at_T(p.eos, rho, T)
    z = np.zeros(X.shape)
    return conserved(p.eos, rho, [z, z], P)


def _modes(g: SplitMix64, count: int, nmax: int):
    out = []
    while len(out) < count:
        nx_, ny_ = g.integer(-nmax, nmax), g.integer(-nmax, nmax)
        if nx_ == 0 and ny_ == 0:
            continue
        out.append((nx_, ny_, g.uniform(0.0, 2.0 * math.pi)))
    return out


def vortex_primitives(p: Problem, strength: float = 5.0, background=(1.0, 0.5, 0.5, 1.0), centre=None):
    """Ideal-gas isentropic (Yee/Shu) vortex of core radius 1 on a uniform background
    (rho, u, v, P); temperature T = P/rho:
      T = T_inf - (gamma-1) s^2 / (8 gamma pi^2) exp(1 - r^2),
      (du, dv) = s / (2 pi) exp((1 - r^2)/2) (-(y - yc), x - xc),
      rho = rho_inf (T/T_inf)^(1/(gamma-1)), P = rho T."""
    gam = p.eos["gamma"]
    X, Y = cell_centres(p)
    if centre is None:
        centre = (0.5 * (p.extent[0] + p.extent[1]), 0.5 * (p.extent[2] + p.extent[3]))
    rho_inf, u_inf, v_inf, P_inf = background
    T_inf = P_inf / rho_inf
    dx_, dy_ = X - centre[0], Y - centre[1]
    r2 = dx_ * dx_ + dy_ * dy_
    T = T_inf - (gam - 1.0) * strength ** 2 / (8.0 * gam * math.pi ** 2) * np.exp(1.0 - r2)
    rho = rho_inf * (T / T_inf) ** (1.0 / (gam - 1.0))
    amp = strength / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
    u = u_inf - amp * dy_
    v = v_inf + amp * dx_
    return rho, u, v, rho * T


def vortex_acoustic_2d(p: Problem = VORTEX_SCALE_2D, seed: int = 4, amp: float = 1e-3, waves: int = 8) -> np.ndarray:
    """Isentropic vortex plus `waves` seeded acoustic plane waves with integer modes
    |n_x|, |n_y| <= 8: dP = amp P_inf cos(2 pi n.x / L + phi) / waves, drho = dP / c_inf^2,
    du = dP / (rho_inf c_inf) n/|n|."""
    rho, u, v, P = vortex_primitives(p)
    gam = p.eos["gamma"]
    rho_inf, P_inf = 1.0, 1.0
    c_inf = math.sqrt(gam * P_inf / rho_inf)
    X, Y = cell_centres(p)
    L = p.extent[1] - p.extent[0]
    g = SplitMix64(seed)
    for nx_, ny_, phi in _modes(g, waves, 8):
        dP = amp * P_inf * np.cos(2.0 * math.pi * (nx_ * X + ny_ * Y) / L + phi) / waves
        nn = math.hypot(nx_, ny_)
        P = P + dP
        rho = rho + dP / c_inf ** 2
        u = u + dP / (rho_inf * c_inf) * nx_ / nn
        v = v + dP / (rho_inf * c_inf) * ny_ / nn
    return conserved(p.eos, rho, [u, v], P)


def vortex_density_2d(p: Problem = VORTEX_ADJOINT_2D, seed: int = 5, amp: float = 1e-2, modes: int = 8) -> np.ndarray:
    """Isentropic vortex with the density multiplied by 1 + amp * mean_m cos(2 pi n.x / L + phi_m)
    at fixed pressure, integer modes |n_x|, |n_y| <= 8."""
    rho, u, v, P = vortex_primitives(p)
    X, Y = cell_centres(p)
    L = p.extent[1] - p.extent[0]
    g = SplitMix64(seed)
    pert = np.zeros(X.shape)
    for nx_, ny_, phi in _modes(g, modes, 8):
        pert += np.cos(2.0 * math.pi * (nx_ * X + ny_ * Y) / L + phi)
    rho = rho * (1.0 + amp * pert / modes)
    return conserved(p.eos, rho, [u, v], P)


def objective_weight(p: Problem = VORTEX_ADJOINT_2D, seed: int = 50, modes: int = 4) -> np.ndarray:
    """Smooth weight g(x) = 1 + 1/2 mean_m cos(2 pi n.x / L + phi_m), |n_x|, |n_y| <= 3; shape (ny, nx)."""
    X, Y = cell_centres(p)
    L = p.extent[1] - p.extent[0]
    g = SplitMix64(seed)
    acc = np.zeros(X.shape)
    for nx_, ny_, phi in _modes(g, modes, 3):
        acc += np.cos(2.0 * math.pi * (nx_ * X + ny_ * Y) / L + phi)
    return np.ascontiguousarray(1.0 + 0.5 * acc / modes)


def directions(p: Problem, count: int = 20, seed: int = 500, modes: int = 4) -> np.ndarray:
    """`count` smooth perturbation fields of the initial W, each a sum of `modes` seeded Fourier
    modes (|n_x|, |n_y| <= 4) per component, scaled to unit RMS over all components and cells;
    shape (count, D+2, ny, nx)."""
    X, Y = cell_centres(p)
    L = p.extent[1] - p.extent[0]
    nc = p.dim + 2
    g = SplitMix64(seed)
    out = np.zeros((count, nc) + X.shape)
    for d in range(count):
        for k in range(nc):
            for nx_, ny_, phi in _modes(g, modes, 4):
                out[d, k] += np.cos(2.0 * math.pi * (nx_ * X + ny_ * Y) / L + phi)
        out[d] /= math.sqrt(np.mean(out[d] ** 2))
    return out


def argrow_1d(case: dict, n: int = 1000) -> Problem:
    """One of the van der Waals shock tubes of Sec. IV D (table of three cases): reduced units
    a = 3, b = 1/3, R = 1, cv = R / (R/cv) of the case, x in [0, 1], CFL 0.8, run to the case's
    t_end.  `case` holds the table's row: R_over_cv, rhoL, PL, rhoR, PR, t_end."""
    eos = {"kind": "vdw", "a": 3.0, "b": 1.0 / 3.0, "R": 1.0, "cv": 1.0 / case["R_over_cv"]}
    return Problem(f"argrow_{case['case']}_1d_{n}", 1, n, 1, (0.0, 1.0, 0.0, 0.0), ZG, eos, 0.8, case["t_end"], 0)


def argrow_states(case: dict):
    """(rho, u, P) left and right of the diaphragm at x = 0.5 (u = 0 on both sides)."""
    return (case["rhoL"], 0.0, case["PL"]), (case["rhoR"], 0.0, case["PR"])


def shu_osher_1d(p: Problem = SHU_OSHER_1D) -> np.ndarray:
    """Shu-Osher shock / entropy-wave interaction (Sec. IV B): the post-shock state of a Mach 3
    shock for x < -4, a sinusoidal density field 1 + 0.2 sin(5x) at rest with P = 1 ahead of it."""
    X, _ = cell_centres(p)
    L = X < -4.0
    rho = np.where(L, 3.857143, 1.0 + 0.2 * np.sin(5.0 * X))
    u = np.where(L, 2.629369, 0.0)
    P = np.where(L, 10.33333, 1.0)
    return conserved(p.eos, rho, [u], P)


def gresho_primitives(p: Problem = GRESHO_2D, P0: float = 5.0):
    """Exact steady Gresho vortex (Sec. IV A) about the domain centre: rho = 1, u_phi = 5r (r < 0.2),
    2 - 5r (0.2 <= r < 0.4), 0 beyond; P = P0 + 12.5 r^2, + 4 (1 - 5r - ln 0.2 + ln r) in the ring,
    P0 - 2 + 4 ln 2 outside.  Returns rho, u, v, P."""
    X, Y = cell_centres(p)
    x0, x1, y0, y1 = p.extent
    dx_, dy_ = X - 0.5 * (x0 + x1), Y - 0.5 * (y0 + y1)
    r = np.hypot(dx_, dy_)
    rs = np.maximum(r, 1e-300)
    uphi = np.where(r < 0.2, 5.0 * r, np.where(r < 0.4, 2.0 - 5.0 * r, 0.0))
    ring = P0 + 12.5 * r * r + 4.0 * (1.0 - 5.0 * r - math.log(0.2) + np.log(rs))
    P = np.where(r < 0.2, P0 + 12.5 * r * r, np.where(r < 0.4, ring, P0 - 2.0 + 4.0 * math.log(2.0)))
    u = np.where(r > 0.0, -uphi * dy_ / rs, 0.0)
    v = np.where(r > 0.0, uphi * dx_ / rs, 0.0)
    return np.ones_like(X), u, v, P


def gresho_2d(p: Problem = GRESHO_2D) -> np.ndarray:
    rho, u, v, P = gresho_primitives(p)
    return conserved(p.eos, rho, [u, v], P)


_SHOCK_VORTEX_FILE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                                  "shock_vortex.json")


def shock_vortex_setup(p: Problem) -> dict:
    """The stored set-up of the shock-vortex case whose EOS p has (written by the fixture script
    beside the file, from the oracle's normal-shock and vortex-shooting routines): upstream and
    downstream (rho, u, P), the vortex profile rho(r), P(r) on r = j dr, and the geometry."""
    with open(_SHOCK_VORTEX_FILE) as fh:
        d = json.load(fh)
    key = "ideal" if p.eos["kind"] == "ideal" else "bzt"
    if d[key]["eos"] != p.eos:
        raise ValueError(f"no stored shock-vortex set-up for the EOS {p.eos}")
    return {**d, **d[key]}


def inflow_state(p: Problem) -> np.ndarray:
    """Conserved state W_in held by the pinned-inflow ghost cells (the upstream shock state)."""
    rho1, u1, P1 = shock_vortex_setup(p)["upstream"]
    return conserved(p.eos, np.array(rho1), [np.array(u1), np.array(0.0)], np.array(P1)).reshape(-1)


def shock_vortex_2d(p: Problem = SHOCK_VORTEX_IDEAL) -> np.ndarray:
    """Upstream state plus the isentropic vortex for x < x_s, downstream state for x >= x_s; the
    vortex's rho(r) and P(r) are interpolated linearly from the stored profile (ambient beyond it),
    its velocity u_phi(r) = beta_v/(2 pi R_c) r exp((1 - r^2/R_c^2)/2) is added to (u1, 0)."""
    d = shock_vortex_setup(p)
    X, Y = cell_centres(p)
    (rho1, u1, P1), (rho2, u2, P2) = d["upstream"], d["downstream"]
    xc, yc = d["vortex_centre"]
    bv, Rc = d["beta_v"], d["Rc"]
    dxv, dyv = X - xc, Y - yc
    r = np.hypot(dxv, dyv)
    rr = np.arange(len(d["profile_rho"])) * d["profile_dr"]
    rho_v = np.interp(r, rr, d["profile_rho"], right=rho1)
    P_v = np.interp(r, rr, d["profile_P"], right=P1)
    amp = bv / (2.0 * math.pi * Rc) * np.exp(0.5 * (1.0 - (r / Rc) ** 2))  # u_phi / r
    up = X < d["x_shock"]
    rho = np.where(up, rho_v, rho2)
    P = np.where(up, P_v, P2)
    u = np.where(up, u1 - amp * dyv, u2)
    v = np.where(up, amp * dxv, 0.0)
    return conserved(p.eos, rho, [u, v], P)


def initial_field(p: Problem) -> np.ndarray:
    """W0 of a named problem at its (possibly resized) grid."""
    base = p.name.split("@")[0]
    if base.startswith("sod_1d"):
        return sod_1d(p)
    if base.startswith("strong_shock_1d"):
        return sod_1d(p, left=(1.0, 0.0, 1000.0), right=(1.0, 0.0, 0.01))
    if base.startswith("shu_osher_1d"):
        return shu_osher_1d(p)
    if base.startswith("gresho_2d"):
        return gresho_2d(p)
    if base.startswith("quadrants_2d"):
        return quadrants_2d(p)
    if base.startswith("bzt_interface_2d") or base.startswith("bzt_interface_cvt_2d"):
        return bzt_interface_2d(p)
    if base.startswith("vortex_acoustic_2d"):
        return vortex_acoustic_2d(p)
    if base.startswith("vortex_adjoint_2d"):
        return vortex_density_2d(p)
    if base.startswith("shock_vortex"):
        return shock_vortex_2d(p)
    raise KeyError(p.name)
