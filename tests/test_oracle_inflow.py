"""Pins of the shock-vortex set-up (Sec. IV H) and of the oracle's pinned-inflow boundary.  CPU only.

* The stationary normal shock from the mass, momentum and stagnation-enthalpy jumps: the textbook
  ideal-gas relations and the paper's printed states (ideal gas and BZT van der Waals gas).
* The vortex by RK2 shooting along the ambient isentrope: the closed-form Yee/Shu vortex for the
  ideal gas; for the van der Waals gas the polytropic isentrope T (1/rho - b)^(R/cv) = const and the
  radial balance dP/dr = rho u_phi^2 / r.
* The stored set-up file equals a fresh run of its fixture script.
* The pinned-inflow side: a uniform state equal to the pinned one is a fixed point; at beta = 1/2
  one step is the Lax-Friedrichs update with the ghost column holding W_in; the sensor sees the
  ghost column's flux and velocity (closed form at a jump between W_in and the interior).
"""
import json
import math
import os
import sys

import numpy as np
import pytest

from oracle import oracle as O
from oracle import shock_vortex as SV
from paper_2609_10639_b300 import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "paper_numbers.json")))
SVJ = json.load(open(os.path.join(HERE, "golden", "shock_vortex.json")))
BZT = {"kind": "vdw", "a": 1.0, "b": 0.3, "R": 1.0, "cv": 50.0}


def printed(x, ref, digits):
    """x rounds to the printed value `ref` (given to `digits` decimals)."""
    return abs(x - ref) <= 0.5 * 10.0 ** (-digits) + 1e-12


def test_ideal_normal_shock_matches_textbook_relations_and_printed_state():
    g = GOLD["ideal_normal_shock"]
    gam, M = g["gamma"], g["Ms"]
    (r1, u1, P1), (r2, u2, P2) = SV.normal_shock({"kind": "ideal", "gamma": gam}, 1.0, 1.0, M)
    # textbook Rankine-Hugoniot relations of a normal shock
    assert u1 == pytest.approx(M * math.sqrt(gam), rel=1e-14)
    assert r2 == pytest.approx((gam + 1) * M * M / ((gam - 1) * M * M + 2), rel=1e-12)
    assert P2 == pytest.approx(1 + 2 * gam / (gam + 1) * (M * M - 1), rel=1e-12)
    assert u2 == pytest.approx(u1 / r2, rel=1e-12)
    for x, key in [(u1, "u1"), (r2, "rho2"), (u2, "u2"), (P2, "P2")]:
        assert printed(x, g[key], 3), (key, x)


def test_bzt_normal_shock_matches_printed_state():
    # Sec. IV H prints the BZT shock at M_s = 1.2 from rho1 = 0.70, P1 = 0.3787 (T1 ~ 0.980):
    # rho2 = 1.506, u2 = 0.251, P2 = 0.488, Gamma2 = +4.47, Gamma1 = -0.255, c_s1 = 0.4497.
    g = GOLD["bzt_normal_shock"]
    (r1, u1, P1), (r2, u2, P2) = SV.normal_shock(BZT, g["rho1"], g["P1"], g["Ms"])
    assert printed(r2, g["rho2"], 3) and printed(u2, g["u2"], 3) and printed(P2, g["P2"], 3), (r2, u2, P2)
    e1 = SV.energy_from_pressure(BZT, r1, P1)
    e2 = SV.energy_from_pressure(BZT, r2, P2)
    assert printed(O.fundamental_derivative(BZT, r2, e2), g["Gamma2"], 2)
    # Gamma1 = -0.2545 at this state: printed as -0.255, within one unit of the third digit
    assert abs(O.fundamental_derivative(BZT, r1, e1) - GOLD["bzt_ambient"]["Gamma"]) <= 1e-3
    assert abs(u1 / g["Ms"] - g["cs1"]) <= 2e-4
    # the jump carries the same flux on both sides (Eqs. 9-10, the oracle's flux): mass, momentum
    # and energy flux (rho E + P) u = rho u (h + u^2/2)
    W1 = wl.conserved(BZT, np.array(r1), [np.array(u1)], np.array(P1)).ravel()
    W2 = wl.conserved(BZT, np.array(r2), [np.array(u2)], np.array(P2)).ravel()
    np.testing.assert_allclose(O.flux(1, BZT, W1)[0], O.flux(1, BZT, W2)[0], rtol=2e-13)


def test_vortex_shooting_reduces_to_the_closed_form_ideal_vortex():
    # ideal gas, rho_inf = P_inf = 1: T = 1 - (gamma-1) beta_v^2/(8 gamma pi^2) exp(1 - r^2),
    # rho = T^(1/(gamma-1)), P = rho T (the classical Yee/Shu vortex)
    gam, bv = 1.4, 2.0
    errs = []
    for n in (12000, 24000):
        r, rho, e, P = SV.vortex_profile({"kind": "ideal", "gamma": gam}, 1.0, 1.0, beta_v=bv, r_max=12.0, n=n)
        T = 1.0 - (gam - 1.0) * bv * bv / (8.0 * gam * math.pi ** 2) * np.exp(1.0 - r * r)
        errs.append(max(np.abs(rho - T ** (1.0 / (gam - 1.0))).max(), np.abs(P - T ** (gam / (gam - 1.0))).max()))
    assert errs[1] < 1e-8
    assert 3.5 < errs[0] / errs[1] < 4.5  # the integration is second order (Heun's RK2)
    # a wrong exponent or factor in u_phi is visible at the core (rho(0) ~ 0.93)
    assert abs(rho[0] - (1.0 - (gam - 1.0) * bv * bv / (8.0 * gam * math.pi ** 2) * math.e) ** 2.5) < 1e-8


def test_vdw_vortex_is_isentropic_and_in_radial_balance():
    r, rho, e, P = SV.vortex_profile(BZT, 0.7, 0.3787, beta_v=2.0, r_max=12.0, n=24000)
    a, b, R, cv = BZT["a"], BZT["b"], BZT["R"], BZT["cv"]
    T = (e + a * rho) / cv
    inv = T * (1.0 / rho - b) ** (R / cv)  # constant along a polytropic van der Waals isentrope
    np.testing.assert_allclose(inv, inv[-1], rtol=1e-9)
    # dP/dr = rho u_phi^2 / r (central differences of the integrated profile)
    h = r[1] - r[0]
    dPdr = (P[2:] - P[:-2]) / (2 * h)
    rhs = rho[1:-1] * SV.u_phi(r[1:-1]) ** 2 / r[1:-1]
    assert np.abs(dPdr - rhs).max() <= 1e-6 * np.abs(rhs).max()
    assert rho[0] < 0.5  # centrifugal rarefaction of the core (Sec. IV H): ~0.451


def test_stored_set_up_equals_its_fixture_script():
    sys.path.insert(0, os.path.join(HERE, "golden"))
    import make_shock_vortex

    fresh = make_shock_vortex.make()
    for key in ("ideal", "bzt"):
        np.testing.assert_allclose(SVJ[key]["upstream"], fresh[key]["upstream"], rtol=1e-14)
        np.testing.assert_allclose(SVJ[key]["downstream"], fresh[key]["downstream"], rtol=1e-14)
        np.testing.assert_allclose(SVJ[key]["profile_rho"], fresh[key]["profile_rho"], rtol=1e-13)
        np.testing.assert_allclose(SVJ[key]["profile_P"], fresh[key]["profile_P"], rtol=1e-13)
    for k in ("domain", "x_shock", "vortex_centre", "beta_v", "Rc", "Ms", "profile_dr"):
        assert SVJ[k] == fresh[k]


# --------------------------------------------------------------------------------------------
# The pinned-inflow side (x-lo): ghost cells hold W_in
def _inflow_problem(nx=24, ny=10):
    return wl.Problem("inflow_test", 2, nx, ny, (0.0, 1.0, 0.0, ny / nx), wl.INFLOW_BC, wl.IDEAL14, 0.5, 0.0, 0)


def test_uniform_pinned_state_is_a_fixed_point():
    p = _inflow_problem()
    W = wl.conserved(p.eos, np.array(1.2), [np.array(0.9), np.array(0.2)], np.array(0.8)).reshape(-1)
    W0 = np.ascontiguousarray(np.broadcast_to(W.reshape(4, 1, 1), (4, p.ny, p.nx)))
    s = O.OracleSolver(2, p.nx, p.ny, p.dx, p.bc, p.eos)
    s.set_inflow(W)
    s.init(W0)
    s.step(300)
    np.testing.assert_allclose(s.W(), W0, rtol=1e-13)
    assert np.all(s.beta() == 1.0)


def test_half_beta_step_with_pinned_inflow_is_lax_friedrichs():
    # beta = 1/2: post-collision populations are the equilibrium everywhere, the ghost's too
    # (f*_{x+}(-1) = W_in/4 + Q_in,x/(2c)), so one step is Lax-Friedrichs with W(-1) = W_in.
    p = _inflow_problem(20, 12)
    rng = np.random.default_rng(7)
    rho = 1.0 + 0.3 * rng.random((p.ny, p.nx))
    u, v = 0.8 + 0.2 * rng.random((p.ny, p.nx)), 0.3 * rng.standard_normal((p.ny, p.nx))
    P = 1.0 + 0.3 * rng.random((p.ny, p.nx))
    W = wl.conserved(p.eos, rho, [u, v], P)
    Win = wl.conserved(p.eos, np.array(1.1), [np.array(1.0), np.array(0.0)], np.array(0.9)).reshape(-1)
    s = O.OracleSolver(2, p.nx, p.ny, p.dx, p.bc, p.eos, beta_mode="const", beta_const=0.5)
    s.set_inflow(Win)
    s.init(W)
    s.step(1)
    gam = p.eos["gamma"]

    def flux(Wf):
        r_, ux, uy = Wf[0], Wf[1] / Wf[0], Wf[2] / Wf[0]
        Pf = (gam - 1.0) * (Wf[3] - 0.5 * r_ * (ux * ux + uy * uy))
        return (np.stack([Wf[1], Wf[1] * ux + Pf, Wf[2] * ux, (Wf[3] + Pf) * ux]),
                np.stack([Wf[2], Wf[1] * uy, Wf[2] * uy + Pf, (Wf[3] + Pf) * uy]), ux, uy, np.sqrt(gam * Pf / r_))

    Qx, Qy, ux, uy, cs = flux(W)
    c = max(float((np.abs(ux) + cs).max()), float((np.abs(uy) + cs).max())) / p.cfl
    Qin = flux(Win.reshape(4, 1, 1))[0][:, :, 0]  # (4, 1)
    ghostW = np.broadcast_to(Win.reshape(4, 1, 1), (4, p.ny, 1))
    ghostQ = np.broadcast_to(Qin.reshape(4, 1, 1), (4, p.ny, 1))
    Wl = np.concatenate([ghostW, W[:, :, :-1]], axis=2)
    Wr = np.concatenate([W[:, :, 1:], W[:, :, -1:]], axis=2)  # zero-gradient outflow
    Ql = np.concatenate([ghostQ, Qx[:, :, :-1]], axis=2)
    Qr = np.concatenate([Qx[:, :, 1:], Qx[:, :, -1:]], axis=2)
    ref = (Wl + Wr + np.roll(W, 1, axis=1) + np.roll(W, -1, axis=1)) / 4.0
    ref -= (Qr - Ql) / (2 * c) + (np.roll(Qy, -1, axis=1) - np.roll(Qy, 1, axis=1)) / (2 * c)
    np.testing.assert_allclose(s.W(), ref, rtol=1e-13, atol=1e-13)


def test_sensor_sees_the_ghost_column_at_a_boundary_jump():
    # interior uniform state A, pinned state B, both moving along x: the only jump is between the
    # ghost column and column 0.  s(-1) = s(0) = s_j = (sum_k ((Q_A,k - Q_B,k)/2 / M_k)^2 / 4)^(1/2)
    # with M_k = max_alpha |Q_alpha,k(A)| (interior cells only), s(1) = 0; theta(-1) = theta(0) =
    # d^2/(d^2 + eps) with d = (U_A - U_B)/(2 dx), theta(1) = 0.  So s_bar = (3/4, 1/4, 0) s_j and
    # theta_bar = (3/4, 1/4, 0) theta_j in columns 0, 1, 2, and beta follows Eq. (35).
    p = _inflow_problem(16, 8)
    gam = p.eos["gamma"]
    rA, UA, PA, rB, UB, PB = 1.0, 0.6, 1.0, 1.2, 0.9, 1.3
    WA = wl.conserved(p.eos, np.array(rA), [np.array(UA), np.array(0.0)], np.array(PA)).reshape(-1)
    WB = wl.conserved(p.eos, np.array(rB), [np.array(UB), np.array(0.0)], np.array(PB)).reshape(-1)
    W0 = np.ascontiguousarray(np.broadcast_to(WA.reshape(4, 1, 1), (4, p.ny, p.nx)))
    s = O.OracleSolver(2, p.nx, p.ny, p.dx, p.bc, p.eos, c_sensor=4.0, ducros_eps=1e-6)
    s.set_inflow(WB)
    s.init(W0)
    F = s.sensor_fields()

    def Qx(r_, U, P_):
        E = P_ / (gam - 1.0) + 0.5 * r_ * U * U
        return np.array([r_ * U, r_ * U * U + P_, 0.0, (E + P_) * U])

    QA, QB = Qx(rA, UA, PA), Qx(rB, UB, PB)
    M = np.array([abs(QA[0]), QA[1], PA, abs(QA[3])])  # Q_y(A) = (0, 0, P_A, 0)
    sj = math.sqrt(np.sum(((QA - QB) / 2.0 / M) ** 2) / 4.0)
    d = (UA - UB) / (2.0 * p.dx)
    tj = d * d / (d * d + 1e-6)
    for col, w in ((0, 0.75), (1, 0.25), (2, 0.0)):
        np.testing.assert_allclose(F["s_bar"][:, col], w * sj, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(F["theta_bar"][:, col], w * tj, rtol=1e-12, atol=1e-15)
        chi = min(max(4.0 * w * sj * w * tj, 0.0), 1.0)
        np.testing.assert_allclose(F["beta"][:, col], 1.0 - 0.25 * chi, rtol=0, atol=1e-14)
    assert F["beta"][0, 0] < 1.0 - 1e-3
