"""ORACLE: test infrastructure only.  Exact solution of the 1D ideal-gas Riemann problem.

Used to pin the oracle's 1D two-state run (density L1 error against the exact self-similar
solution).  Written from the gas-dynamics of a single-component ideal gas (P = (gamma-1) rho e,
Eq. 15): the star pressure p* is the root of the pressure function
    f(p) = f_L(p) + f_R(p) + (u_R - u_L),
    f_K(p) = (p - p_K) sqrt(A_K / (p + B_K)),                 p > p_K  (shock),
             2 a_K / (gamma-1) ((p/p_K)^((gamma-1)/(2 gamma)) - 1), p <= p_K (rarefaction),
    A_K = 2 / ((gamma+1) rho_K),  B_K = (gamma-1)/(gamma+1) p_K,  a_K^2 = gamma p_K / rho_K,
and u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2.  The solution is then sampled along
xi = (x - x0)/t through the left wave, the contact at u* and the right wave.
Two independent root-finders (Newton and bisection) are provided so that a test can check
that they agree.
"""
from __future__ import annotations

import math

import numpy as np


def _fk(p, rho, pk, gam):
    a = math.sqrt(gam * pk / rho)
    if p > pk:
        A = 2.0 / ((gam + 1.0) * rho)
        B = (gam - 1.0) / (gam + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (B + p))
    r = p / pk
    return (2.0 * a / (gam - 1.0) * (r ** ((gam - 1.0) / (2.0 * gam)) - 1.0),
            1.0 / (rho * a) * r ** (-(gam + 1.0) / (2.0 * gam)))


def _pressure_fn(p, L, R, gam):
    fl, dl = _fk(p, L[0], L[2], gam)
    fr, dr = _fk(p, R[0], R[2], gam)
    return fl + fr + (R[1] - L[1]), dl + dr


def star_state_newton(L, R, gam, tol=1e-15, maxit=200):
    """p*, u* by Newton iteration on the pressure function from the two-rarefaction guess."""
    aL, aR = math.sqrt(gam * L[2] / L[0]), math.sqrt(gam * R[2] / R[0])
    z = (gam - 1.0) / (2.0 * gam)
    p = ((aL + aR - 0.5 * (gam - 1.0) * (R[1] - L[1])) / (aL / L[2] ** z + aR / R[2] ** z)) ** (1.0 / z)
    p = max(p, 1e-14)
    for _ in range(maxit):
        f, df = _pressure_fn(p, L, R, gam)
        pn = max(p - f / df, 1e-14)
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, L[0], L[2], gam)
    fr, _ = _fk(p, R[0], R[2], gam)
    return p, 0.5 * (L[1] + R[1]) + 0.5 * (fr - fl)


def star_state_bisection(L, R, gam):
    """p*, u* by bisection on the (monotone increasing) pressure function."""
    lo, hi = 1e-14, 1.0
    while _pressure_fn(hi, L, R, gam)[0] < 0.0:
        hi *= 2.0
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        if _pressure_fn(mid, L, R, gam)[0] < 0.0:
            lo = mid
        else:
            hi = mid
        if hi - lo <= 1e-16 * hi:
            break
    p = 0.5 * (lo + hi)
    fl, _ = _fk(p, L[0], L[2], gam)
    fr, _ = _fk(p, R[0], R[2], gam)
    return p, 0.5 * (L[1] + R[1]) + 0.5 * (fr - fl)


def sample(xi, L, R, gam, ps, us):
    """(rho, u, p) of the self-similar solution at xi = (x - x0)/t."""
    g1 = (gam - 1.0) / (gam + 1.0)
    if xi <= us:  # left of the contact
        rho, u, p = L
        a = math.sqrt(gam * p / rho)
        if ps > p:  # left shock
            S = u - a * math.sqrt((gam + 1.0) / (2.0 * gam) * ps / p + (gam - 1.0) / (2.0 * gam))
            if xi <= S:
                return rho, u, p
            return rho * (ps / p + g1) / (g1 * ps / p + 1.0), us, ps
        a_star = a * (ps / p) ** ((gam - 1.0) / (2.0 * gam))
        if xi <= u - a:
            return rho, u, p
        if xi >= us - a_star:
            return rho * (ps / p) ** (1.0 / gam), us, ps
        uf = 2.0 / (gam + 1.0) * (a + 0.5 * (gam - 1.0) * u + xi)
        af = 2.0 / (gam + 1.0) * (a + 0.5 * (gam - 1.0) * (u - xi))
        return rho * (af / a) ** (2.0 / (gam - 1.0)), uf, p * (af / a) ** (2.0 * gam / (gam - 1.0))
    rho, u, p = R
    a = math.sqrt(gam * p / rho)
    if ps > p:  # right shock
        S = u + a * math.sqrt((gam + 1.0) / (2.0 * gam) * ps / p + (gam - 1.0) / (2.0 * gam))
        if xi >= S:
            return rho, u, p
        return rho * (ps / p + g1) / (g1 * ps / p + 1.0), us, ps
    a_star = a * (ps / p) ** ((gam - 1.0) / (2.0 * gam))
    if xi >= u + a:
        return rho, u, p
    if xi <= us + a_star:
        return rho * (ps / p) ** (1.0 / gam), us, ps
    uf = 2.0 / (gam + 1.0) * (-a + 0.5 * (gam - 1.0) * u + xi)
    af = 2.0 / (gam + 1.0) * (a - 0.5 * (gam - 1.0) * (u - xi))
    return rho * (af / a) ** (2.0 / (gam - 1.0)), uf, p * (af / a) ** (2.0 * gam / (gam - 1.0))


def solution(x, t, L, R, gam, x0=0.5):
    """Arrays rho, u, p at positions x and time t > 0."""
    ps, us = star_state_newton(L, R, gam)
    out = np.array([sample((xx - x0) / t, L, R, gam, ps, us) for xx in np.asarray(x).ravel()])
    return out[:, 0], out[:, 1], out[:, 2]
