"""Pins of the oracle's thermodynamics (Sec. II C) against the paper's printed numbers,
closed forms and finite-difference definitions.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2609_10639_b300 import workloads as wl

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def bzt_eos():
    g = GOLD["bzt_vdw_eos"]
    return {"kind": "vdw", "a": g["a"], "b": g["b"], "R": g["R"], "cv": g["R"] / (g["gamma"] - 1.0)}


def close(x, ref, digits_ref):
    """Agreement to the digits the paper prints: within one unit of the last printed place (the
    paper sometimes truncates, e.g. c_s0 = 0.44978 printed as 0.4497)."""
    s = repr(digits_ref)
    dec = len(s.split(".")[1]) if "." in s else 0
    return abs(x - ref) <= 10 ** (-dec) + 1e-12


def test_ideal_sound_speed_closed_form():
    # Eq. (15): c_s^2 = gamma (gamma - 1) e, P = (gamma - 1) rho e.
    eos = wl.IDEAL14
    for rho, e in [(1.0, 2.5), (0.125, 2.0), (3.0, 0.1)]:
        P, cs2 = O.eos_eval(eos, rho, e)
        assert P == pytest.approx(0.4 * rho * e, rel=1e-15)
        assert cs2 == pytest.approx(1.4 * 0.4 * e, rel=1e-15)


@pytest.mark.parametrize("eos", [wl.IDEAL14, wl.VDW_REDUCED, bzt_eos()], ids=["ideal", "vdw_reduced", "vdw_bzt"])
def test_sound_speed_matches_definition_by_finite_differences(eos):
    # Eq. (13): c_s^2 = P_rho|_e + P/rho^2 P_e|_rho, checked against central differences of the
    # oracle's own P(rho, e) (an error in the chain rule for the vdW closure fails this).
    rng = np.random.default_rng(0)
    for _ in range(50):
        if eos["kind"] == "ideal":
            rho, e = rng.uniform(0.1, 3.0), rng.uniform(0.1, 5.0)
        else:
            rho = rng.uniform(0.3, 1.2) / (3.0 * eos["b"]) * 1.0
            rho = min(rho, 0.9 / eos["b"])
            T = rng.uniform(1.0, 1.5) * 8.0 * eos["a"] / (27.0 * eos["b"] * eos["R"])
            e = eos["cv"] * T - eos["a"] * rho
        P, cs2 = O.eos_eval(eos, rho, e)
        h = 1e-5
        P_rho = (O.eos_eval(eos, rho + h, e)[0] - O.eos_eval(eos, rho - h, e)[0]) / (2 * h)
        P_e = (O.eos_eval(eos, rho, e + h)[0] - O.eos_eval(eos, rho, e - h)[0]) / (2 * h)
        assert cs2 == pytest.approx(P_rho + P / rho ** 2 * P_e, rel=1e-7, abs=1e-9)


def test_vdw_critical_point():
    # Sec. IV F: rho_c = 1.111, T_c = 0.988, P_c = 0.412 for a = 1, b = 0.3, R = 1.  At the
    # critical point (dP/drho)_T = (d2P/drho2)_T = 0; derivatives of the oracle's P along the
    # isotherm e = cv T - a rho by central differences.
    eos = bzt_eos()
    cp = GOLD["bzt_critical_point"]
    rc, Tc = 1.0 / (3.0 * eos["b"]), 8.0 * eos["a"] / (27.0 * eos["b"] * eos["R"])
    assert close(rc, cp["rho"], cp["rho"]) and close(Tc, cp["T"], cp["T"])
    P_of = lambda r: O.eos_eval(eos, r, eos["cv"] * Tc - eos["a"] * r)[0]
    assert close(P_of(rc), cp["P"], cp["P"])
    h = 1e-4
    d1 = (P_of(rc + h) - P_of(rc - h)) / (2 * h)
    d2 = (P_of(rc + h) - 2 * P_of(rc) + P_of(rc - h)) / h ** 2
    assert abs(d1) < 1e-7 and abs(d2) < 1e-4


def test_bzt_ambient_state():
    # Secs. IV G-H: rho0 = 0.70, T = 0.980 gives P0 = 0.3787, c_s0 = 0.4497, Gamma0 = -0.255.
    eos = bzt_eos()
    g = GOLD["bzt_ambient"]
    e = wl.internal_energy(eos, g["rho"], g["P"])
    T = (e + eos["a"] * g["rho"]) / eos["cv"]
    assert close(T, g["T"], g["T"])
    P, cs2 = O.eos_eval(eos, g["rho"], eos["cv"] * g["T"] - eos["a"] * g["rho"])
    assert abs(P - g["P"]) / g["P"] < 1e-3  # T printed to 3 digits
    P, cs2 = O.eos_eval(eos, g["rho"], e)
    assert P == pytest.approx(g["P"], rel=1e-14)
    assert close(math.sqrt(cs2), g["cs"], g["cs"])
    assert close(O.fundamental_derivative(eos, g["rho"], e), g["Gamma"], g["Gamma"])


def _isentrope(eos, rho0, P0, targets, h=1e-4):
    """Classical RK4 along de/drho = P/rho^2 (T ds = de - P/rho^2 drho = 0) using the oracle's P."""
    e, r, out = wl.internal_energy(eos, rho0, P0), rho0, {}
    f = lambda rr, ee: O.eos_eval(eos, rr, ee)[0] / rr ** 2
    for tgt in sorted(targets):
        while r < tgt - 1e-13:
            hh = min(h, tgt - r)
            k1 = f(r, e)
            k2 = f(r + hh / 2, e + hh / 2 * k1)
            k3 = f(r + hh / 2, e + hh / 2 * k2)
            k4 = f(r + hh, e + hh * k3)
            e += hh / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
            r += hh
        out[tgt] = (math.sqrt(O.eos_eval(eos, r, e)[1]), O.fundamental_derivative(eos, r, e))
    return out


def test_isentropes():
    # Sec. IV G: along the ambient isentrope c_s falls 0.450 -> 0.246 (BZT gas, minimum near
    # rho 1.0-1.1) but rises 0.450 -> 0.501 for the ideal gas with the same ambient sound speed.
    g = GOLD["bzt_isentrope_cs"]
    rhos = list(np.arange(0.70, 1.2001, 0.01).round(6))
    res = _isentrope(bzt_eos(), 0.70, GOLD["bzt_ambient"]["P"], rhos)
    for r, cs in zip(g["rho"], g["cs"]):
        assert close(res[round(r, 6)][0], cs, cs)
    rmin = min(res, key=lambda r: res[r][0])
    assert g["min_rho_range"][0] <= rmin <= g["min_rho_range"][1]
    foc = GOLD["bzt_focus_gamma"]
    assert abs(res[foc["rho"]][1] - foc["Gamma"]) < 0.1
    gi = GOLD["ideal_isentrope_cs"]
    P0 = gi["cs0"] ** 2 * gi["rho"][0] / gi["gamma"]
    resi = _isentrope({"kind": "ideal", "gamma": gi["gamma"]}, gi["rho"][0], P0, [gi["rho"][1]])
    assert close(resi[gi["rho"][1]][0], gi["cs"][1], gi["cs"][1])


def test_fundamental_derivative_ideal_closed_form():
    # Gamma = (gamma + 1)/2 for the ideal gas (Secs. IV F-G).
    for gam in (1.4, 5.0 / 3.0, 1.1):
        for rho, e in [(1.0, 2.5), (0.3, 0.7)]:
            assert O.fundamental_derivative({"kind": "ideal", "gamma": gam}, rho, e) == pytest.approx((gam + 1) / 2, rel=1e-13)


def test_fundamental_derivative_matches_finite_difference_along_isentrope():
    eos = bzt_eos()
    rho, P = 0.85, 0.40
    e = wl.internal_energy(eos, rho, P)
    h = 1e-4
    # step along the isentrope to second order: de = P/rho^2 drho
    cs = lambda r, ee: math.sqrt(O.eos_eval(eos, r, ee)[1])
    Pp = O.eos_eval(eos, rho, e)[0]
    ep = e + Pp / rho ** 2 * h
    em = e - Pp / rho ** 2 * h
    # second-order correction of the isentrope: d2e/drho2 = d(P/rho^2)/drho along it
    dPr = (O.eos_eval(eos, rho + 1e-6, e)[0] - O.eos_eval(eos, rho - 1e-6, e)[0]) / 2e-6
    dPe = (O.eos_eval(eos, rho, e + 1e-6)[0] - O.eos_eval(eos, rho, e - 1e-6)[0]) / 2e-6
    d2 = (dPr + dPe * Pp / rho ** 2) / rho ** 2 - 2 * Pp / rho ** 3
    ep += 0.5 * d2 * h * h
    em += 0.5 * d2 * h * h
    dcs = (cs(rho + h, ep) - cs(rho - h, em)) / (2 * h)
    G_fd = 1 + rho / cs(rho, e) * dcs
    assert O.fundamental_derivative(eos, rho, e) == pytest.approx(G_fd, rel=1e-6)


def test_argrow_and_bzt_gamma_signs():
    # Sec. IV D: Case I lies in Gamma < 0 at both initial states; Cases II and III are classical.
    a = GOLD["argrow_cases"]
    for c in a["cases"]:
        eos = {"kind": "vdw", "a": a["eos"]["a"], "b": a["eos"]["b"], "R": a["eos"]["R"], "cv": a["eos"]["R"] / c["R_over_cv"]}
        for rho, P in [(c["rhoL"], c["PL"]), (c["rhoR"], c["PR"])]:
            e = wl.internal_energy(eos, rho, P)
            assert O.eos_eval(eos, rho, e)[1] > 0
            assert np.sign(O.fundamental_derivative(eos, rho, e)) == c["Gamma_sign"]
    # Eq. (49): the four BZT quadrant states all have Gamma < 0.
    for rho, u, v, P in GOLD["bzt_quadrants"]["states_NE_NW_SW_SE"]:
        assert O.fundamental_derivative(bzt_eos(), rho, wl.internal_energy(bzt_eos(), rho, P)) < 0


def test_bzt_shock_state_gamma():
    g = GOLD["bzt_normal_shock"]
    eos = bzt_eos()
    e2 = wl.internal_energy(eos, g["rho2"], g["P2"])
    assert abs(O.fundamental_derivative(eos, g["rho2"], e2) - g["Gamma2"]) < 0.01  # 4.47 from 3-digit state


def test_stored_bzt_states_are_oracle_accepted():
    # The stored left/right states of the BZT interface input both satisfy the oracle's state
    # rule (c_s^2 > 0 and Gamma < 0) and the flow they start stays hyperbolic in the oracle.
    eos = wl.VDW_REDUCED
    (rl, Pl), (rr, Pr) = wl.bzt_states(3)
    for rho, P in ((rl, Pl), (rr, Pr)):
        e = wl.internal_energy(eos, rho, P)
        assert O.eos_eval(eos, rho, e)[1] > 0 and O.fundamental_derivative(eos, rho, e) < 0
    p = wl.BZT_2D.resized(64)
    s = O.OracleSolver.for_problem(p)
    s.init(wl.bzt_interface_2d(p))
    s.step(10 ** 6, p.t_end)
    assert s.time()[0] == p.t_end
