"""Pins of the oracle's non-polytropic van der Waals gas (a closure admitted by Eq. 11): the
thermal relation of Eq. (16) with a temperature-dependent heat capacity c_v(T) = cv + cv1 T + cv2 T^2,
e = E(T) - a rho, E(T) = cv T + cv1 T^2/2 + cv2 T^3/3, and T(rho, e) by Newton's method.  CPU only.

* With cv1 = cv2 = 0 the Newton inversion reproduces the closed form of the polytropic gas.
* The caloric relation satisfies the consistency condition Eq. (12).
* P(rho, e) round-trips with the forward relation e(rho, P) of the input generator, so the Newton
  root is the temperature of the state.
* c_s^2 equals its definition Eq. (13) by finite differences of P(rho, e).
* The fundamental derivative goes negative (a BZT gas) at the states of the BZT interface input.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2609_10639_b300 import workloads as wl

CVT = wl.VDW_CVT_REDUCED


def random_states(rng, n, rho_range=(0.2, 2.2), T_range=(0.6, 3.0)):
    rho = rng.uniform(*rho_range, n)
    T = rng.uniform(*T_range, n)
    P = wl.vdw_pressure_at_T(CVT, rho, T)
    return rho, T, P


def test_newton_reproduces_the_polytropic_closed_form():
    poly = dict(CVT, cv1=0.0, cv2=0.0)
    ref = {"kind": "vdw", "a": CVT["a"], "b": CVT["b"], "R": CVT["R"], "cv": CVT["cv"]}
    rng = np.random.default_rng(11)
    rho, T, P = random_states(rng, 500)
    for r, p_ in zip(rho, P):
        e = wl.internal_energy(ref, r, p_)
        Pn, cn = O.eos_eval(poly, r, e)
        Pc, cc = O.eos_eval(ref, r, e)
        assert Pn == pytest.approx(Pc, rel=1e-14, abs=1e-14)
        assert cn == pytest.approx(cc, rel=1e-13)


def test_caloric_relation_is_consistent():
    # Eq. (12): (de/drho)_T = [P - T (dP/dT)_rho] / rho^2 (= -a for the van der Waals thermal relation)
    rng = np.random.default_rng(12)
    rho, T, _ = random_states(rng, 200)
    h = 1e-6
    e_of = lambda r, t: wl.internal_energy(CVT, r, wl.vdw_pressure_at_T(CVT, r, t))
    lhs = (e_of(rho + h, T) - e_of(rho - h, T)) / (2 * h)
    dPdT = (wl.vdw_pressure_at_T(CVT, rho, T + h) - wl.vdw_pressure_at_T(CVT, rho, T - h)) / (2 * h)
    rhs = (wl.vdw_pressure_at_T(CVT, rho, T) - T * dPdT) / rho ** 2
    np.testing.assert_allclose(lhs, rhs, rtol=1e-7, atol=1e-7)


def test_pressure_round_trips_through_the_newton_inversion():
    rng = np.random.default_rng(13)
    rho, T, P = random_states(rng, 2000, T_range=(0.3, 8.0))
    for r, p_ in zip(rho, P):
        e = wl.internal_energy(CVT, r, p_)
        Pn, cs2 = O.eos_eval(CVT, r, e)
        assert Pn == pytest.approx(p_, rel=1e-12, abs=1e-13)
        assert np.isfinite(cs2)


def test_sound_speed_is_its_definition():
    # Eq. (13): c_s^2 = (dP/drho)_e + P/rho^2 (dP/de)_rho, by central differences of P(rho, e)
    rng = np.random.default_rng(14)
    rho, T, P = random_states(rng, 300)
    for r, p_ in zip(rho, P):
        e = wl.internal_energy(CVT, r, p_)
        hr, he = 1e-5 * r, 1e-5 * abs(e)
        Pr = (O.eos_eval(CVT, r + hr, e)[0] - O.eos_eval(CVT, r - hr, e)[0]) / (2 * hr)
        Pe = (O.eos_eval(CVT, r, e + he)[0] - O.eos_eval(CVT, r, e - he)[0]) / (2 * he)
        cs2 = O.eos_eval(CVT, r, e)[1]
        assert cs2 == pytest.approx(Pr + p_ / r ** 2 * Pe, rel=2e-7, abs=1e-9)


def test_bzt_interface_states_have_negative_fundamental_derivative():
    # the seeded BZT interface states (accepted for the polytropic gas) stay in the Gamma < 0 region
    # with c_v(T), whose value at the critical temperature is the polytropic 50 R
    for rho, P in wl.bzt_states(3):
        e = wl.internal_energy(CVT, rho, P)
        assert O.eos_eval(CVT, rho, e)[1] > 0.0
        assert O.fundamental_derivative(CVT, rho, e) < 0.0
