"""ORACLE: test infrastructure only (set-up of the shock-vortex interaction, Sec. IV H).

Two EOS-generic constructions the paper states for its shock-vortex case, written with the
oracle's own equation of state (vlbm_oracle.cpp: P(rho, e), c_s^2(rho, e), Sec. II C):

* normal_shock(): the stationary normal shock at upstream Mach number M_s, from the exact jump
  conditions of mass, momentum and stagnation enthalpy across a steady discontinuity
  (rho1 u1 = rho2 u2; P1 + rho1 u1^2 = P2 + rho2 u2^2; h1 + u1^2/2 = h2 + u2^2/2 with h = e + P/rho).
  Eliminating u2 and e2 leaves one equation in rho2, solved by bracketing and Brent's method.
* vortex_profile(): the isentropic vortex with azimuthal velocity
  u_phi(r) = beta_v / (2 pi R_c) r exp((1 - r^2/R_c^2)/2) in radial balance dP/dr = rho u_phi^2 / r,
  integrated inward from the ambient state along its isentrope, de/drho = P/rho^2 (Sec. II C):
  d rho/dr = rho u_phi^2 / (r c_s^2),  de/dr = (P/rho^2) d rho/dr, by Heun's two-stage RK2 (the
  paper's "RK2 shooting").  For the ideal gas it reduces to the closed-form Yee/Shu vortex.

Only the tests and the committed script that writes tests/golden/shock_vortex.json use this.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq

from oracle import oracle as O


def energy_from_pressure(eos: dict, rho: float, P: float) -> float:
    """Specific internal energy e with P(rho, e) = P: the oracle's EOS inverted by Brent's method
    (P is increasing in e at fixed rho for both closures of Sec. II C)."""
    lo, hi = -10.0, 10.0
    while O.eos_eval(eos, rho, lo)[0] > P:
        lo *= 2.0
    while O.eos_eval(eos, rho, hi)[0] < P:
        hi *= 2.0
    return brentq(lambda e: O.eos_eval(eos, rho, e)[0] - P, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=400)


def normal_shock(eos: dict, rho1: float, P1: float, Ms: float):
    """Upstream (rho1, u1, P1) with u1 = M_s c_s1, and the downstream (rho2, u2, P2) of the
    stationary normal shock (mass, momentum and stagnation-enthalpy jumps)."""
    e1 = energy_from_pressure(eos, rho1, P1)
    cs1 = math.sqrt(O.eos_eval(eos, rho1, e1)[1])
    u1 = Ms * cs1
    m = rho1 * u1
    H = e1 + P1 / rho1 + 0.5 * u1 * u1  # stagnation enthalpy

    def residual(rho2):
        u2 = m / rho2
        P2 = P1 + m * (u1 - u2)  # momentum
        e2 = H - 0.5 * u2 * u2 - P2 / rho2  # energy
        return O.eos_eval(eos, rho2, e2)[0] - P2

    # the compressive root: scan upward from just above rho1 for the first sign change
    rmax = (1.0 / eos["b"]) * (1.0 - 1e-9) if eos["kind"] == "vdw" else 50.0 * rho1
    grid = rho1 * (1.0 + np.geomspace(1e-6, rmax / rho1 - 1.0, 4000))
    vals = [residual(r) for r in grid]
    for j in range(len(grid) - 1):
        if vals[j] == 0.0 or vals[j] * vals[j + 1] < 0.0:
            rho2 = brentq(residual, grid[j], grid[j + 1], xtol=1e-15, rtol=1e-15, maxiter=400)
            break
    else:
        raise ValueError("no compressive shock solution found")
    u2 = m / rho2
    P2 = P1 + m * (u1 - u2)
    return (rho1, u1, P1), (rho2, u2, P2)


def u_phi(r, beta_v: float = 2.0, Rc: float = 1.0):
    """Azimuthal velocity of the Yee/Shu vortex profile (Sec. IV H)."""
    return beta_v / (2.0 * math.pi * Rc) * r * np.exp(0.5 * (1.0 - (r / Rc) ** 2))


def vortex_profile(eos: dict, rho_inf: float, P_inf: float, beta_v: float = 2.0, Rc: float = 1.0,
                   r_max: float = 12.0, n: int = 120000):
    """rho(r), e(r), P(r) of the isentropic vortex on r_j = j r_max / n (j = 0..n), integrated
    inward from the ambient (rho_inf, P_inf) at r_max by Heun's RK2."""
    e_inf = energy_from_pressure(eos, rho_inf, P_inf)
    r = np.linspace(0.0, r_max, n + 1)

    def rhs(rr, rho, e):
        if rr == 0.0:  # u_phi^2 / r -> 0 at the axis
            return 0.0, 0.0
        P, cs2 = O.eos_eval(eos, rho, e)
        drho = rho * float(u_phi(rr, beta_v, Rc)) ** 2 / (rr * cs2)
        return drho, P / (rho * rho) * drho

    rho = np.empty(n + 1)
    e = np.empty(n + 1)
    rho[n], e[n] = rho_inf, e_inf
    h = -r_max / n  # inward
    for j in range(n, 0, -1):
        k1 = rhs(r[j], rho[j], e[j])
        k2 = rhs(r[j - 1], rho[j] + h * k1[0], e[j] + h * k1[1])
        rho[j - 1] = rho[j] + 0.5 * h * (k1[0] + k2[0])
        e[j - 1] = e[j] + 0.5 * h * (k1[1] + k2[1])
    P = np.array([O.eos_eval(eos, a, b)[0] for a, b in zip(rho, e)])
    return r, rho, e, P
