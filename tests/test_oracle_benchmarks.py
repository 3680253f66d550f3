"""The oracle's VLBM run against the paper's printed accuracy numbers and claims for its
benchmarks, the 1D ones through the independent reference solver (pinned in
test_oracle_muscl.py):

* the three van der Waals shock tubes of Argrow (Sec. IV D): L1(rho) and L1(P) at N = 1000
  against the reference at N_ref = 3000;
* the strong shock tube (Sec. IV C): L1(rho), L1(u), L1(P) at N = 2000 against N_ref = 4000;
* the Shu-Osher problem (Sec. IV B): the sensor run's L2(rho) against N_ref = 1e4 is about half
  that of the constant beta = 0.9 baseline, both converging at close to first order;
* the Gresho vortex (Sec. IV A, 2D, exact steady solution): the sensor beats the constant
  beta = 0.995 baseline and converges faster.

The paper's numbers come from its own reference solver, whose time step and interface details it
does not give, so each printed value is matched within a factor of 3/2 (soft pins); the measured
ratios are listed beside the readings of the paper.  The reference is compared cell by cell
after averaging its N_ref / N fine cells inside each coarse cell; L1 = dx sum |a - b|,
L2 = (dx sum (a - b)^2)^(1/2).
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2609_10639_b300 import workloads as wl

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))
BAND = 1.5


def primitives(eos, W):
    """rho, u, P of a 1D conserved field (3 x n), P from the oracle's equation of state."""
    rho = W[0]
    u = W[1] / rho
    e = W[2] / rho - 0.5 * u * u
    P = np.array([O.eos_eval(eos, r, ee)[0] for r, ee in zip(rho, e)])
    return rho, u, P


def coarse(a, n):
    return a.reshape(n, -1).mean(axis=1)


def vlbm_run(prob, W0, **over):
    s = O.OracleSolver.for_problem(prob, **over)
    s.init(W0)
    s.step(10 ** 7, prob.t_end)
    assert s.time()[0] == prob.t_end
    return s


def within_band(value, printed):
    return printed / BAND <= value <= printed * BAND


@pytest.mark.parametrize("case", GOLD["argrow_cases"]["cases"], ids=lambda c: c["case"])
def test_argrow_shock_tubes_printed_l1(case):
    n, n_ref = GOLD["argrow_cases"]["N"], GOLD["argrow_cases"]["N_ref"]
    prob = wl.argrow_1d(case, n)
    left, right = wl.argrow_states(case)
    ref_prob = wl.argrow_1d(case, n_ref)
    Wr, _ = O.muscl_1d(prob.eos, wl.sod_1d(ref_prob, left, right)[:, 0, :], ref_prob.dx, "zerograd", prob.t_end)
    s = vlbm_run(prob, wl.sod_1d(prob, left, right))
    rho, _, P = primitives(prob.eos, s.W()[:, 0, :])
    rr, _, Pr = primitives(prob.eos, Wr)
    l1_rho = prob.dx * np.abs(rho - coarse(rr, n)).sum()
    l1_P = prob.dx * np.abs(P - coarse(Pr, n)).sum()
    assert within_band(l1_rho, case["L1_rho_vs_muscl"]), (l1_rho, case["L1_rho_vs_muscl"])
    assert within_band(l1_P, case["L1_P_vs_muscl"]), (l1_P, case["L1_P_vs_muscl"])
    # the sensor marks every discontinuity (Sec. IV D): beta dips below 0.95 somewhere
    assert s.beta().min() < 0.95


def test_strong_shock_tube_printed_l1_against_reference():
    g = GOLD["strong_shock_tube"]
    prob = wl.STRONG_SHOCK_1D
    ref_prob = prob.resized(g["N_ref"])
    left, right = tuple(g["left"]), tuple(g["right"])
    Wr, _ = O.muscl_1d(prob.eos, wl.sod_1d(ref_prob, left, right)[:, 0, :], ref_prob.dx, "zerograd", g["t_end"])
    s = vlbm_run(prob, wl.initial_field(prob))
    a = primitives(prob.eos, s.W()[:, 0, :])
    b = primitives(prob.eos, Wr)
    l1 = [prob.dx * np.abs(x - coarse(y, prob.nx)).sum() for x, y in zip(a, b)]
    for got, key in zip(l1, ("L1_rho_vs_muscl", "L1_u_vs_muscl", "L1_P_vs_muscl")):
        assert within_band(got, g[key]), (key, got, g[key])


@pytest.fixture(scope="module")
def shu_osher_reference():
    g = GOLD["shu_osher"]
    ref_prob = wl.SHU_OSHER_1D.resized(g["N_ref"])
    Wr, _ = O.muscl_1d(ref_prob.eos, wl.shu_osher_1d(ref_prob)[:, 0, :], ref_prob.dx, "zerograd", g["t_end"])
    return Wr[0]


def test_shu_osher_sensor_halves_the_error(shu_osher_reference):
    # beta_max = 0.99: with beta_max = 1 the non-equilibrium start-up pulse of the initial shock
    # travels undamped to the supersonic inflow and changes the inflow state (see the readings)
    g = GOLD["shu_osher"]
    l2 = {}
    for n in (2000, 2500, 5000):
        prob = wl.SHU_OSHER_1D.resized(n)
        W0 = wl.shu_osher_1d(prob)
        ref = coarse(shu_osher_reference, n)
        for mode, over in (("sensor", dict(beta_max=0.99)),
                           ("const", dict(beta_mode="const", beta_const=g["beta_const_baseline"]))):
            rho = vlbm_run(prob, W0, **over).W()[0, 0]
            l2[mode, n] = np.sqrt(prob.dx * np.sum((rho - ref) ** 2))
        assert l2["sensor", n] <= 0.6 * l2["const", n], (n, l2)
    for mode in ("sensor", "const"):
        order = np.log(l2[mode, 2000] / l2[mode, 5000]) / np.log(2.5)
        assert 0.5 < order < 1.5, (mode, order, l2)


def test_gresho_vortex_sensor_against_best_constant_beta():
    # Sec. IV A: the exact steady Gresho vortex to t = 0.5; L2 error of |u| against the exact
    # solution.  The sensor run beats the paper's constant-beta baseline (0.995) at every N and
    # converges faster.  The paper reports close-to-second order for the sensor; the oracle shows
    # 1.3 over N = 64-256 (the kinks of u_phi at r = 0.2, 0.4 limit it; see the readings).
    l2, order = {}, {}
    for mode, over in (("sensor", {}), ("const", dict(beta_mode="const", beta_const=0.995))):
        for n in (64, 128, 256):
            prob = wl.GRESHO_2D.resized(n)
            _, u, v, _ = wl.gresho_primitives(prob)
            W = vlbm_run(prob, wl.gresho_2d(prob), **over).W()
            umag = np.hypot(W[1] / W[0], W[2] / W[0])
            l2[mode, n] = np.sqrt(np.mean((umag - np.hypot(u, v)) ** 2))
        order[mode] = np.log2(l2[mode, 128] / l2[mode, 256])
    for n in (64, 128, 256):
        assert l2["sensor", n] < 0.75 * l2["const", n], l2
    assert order["sensor"] > 1.15 and order["sensor"] > order["const"] + 0.2, order
