"""Closed-form pins of the shock sensor's filter stage (Sec. III D, Eqs. 28-35): the box filter
s_bar = S[s] with weights (1/4, 1/2, 1/4) along each direction, and the Ducros ratio theta with
its filtered value theta_bar = S[theta] (Eq. 33).  CPU only.

The states are built so that every quantity before the filter has an exact value: at constant
velocity and pressure every flux component of an ideal gas is linear in rho, so a density profile
made of two straight pieces that meet at one cell (a slope kink) gives a piecewise-constant
activity s (one value on each side, the mean of the two at the kink cell); a velocity made of two
straight pieces gives exact central differences, hence an exact theta that steps from ~1 to 0
across the kink.  The filter then has a closed-form profile over the three cells around the kink,
which a missing filter, other tap weights, or a filter along the wrong axis all miss.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2609_10639_b300 import workloads as wl

N, I0 = 64, 32  # cells per axis, kink cell
RHO0, U, P0, GAM = 1.0, 0.8, 1.5, 1.4
G1, G2 = 0.5, 2.0  # density slopes left and right of the kink


def kink_profile(v_left, v_kink, v_right):
    """Filter of a profile equal to v_left left of cell I0, v_kink at I0, v_right right of it:
    the closed form of (1/4, 1/2, 1/4) at cells I0-2 .. I0+2."""
    return {
        I0 - 2: v_left,
        I0 - 1: 0.75 * v_left + 0.25 * v_kink,
        I0: 0.25 * v_left + 0.5 * v_kink + 0.25 * v_right,
        I0 + 1: 0.25 * v_kink + 0.75 * v_right,
        I0 + 2: v_right,
    }


def density_kink(dx):
    j = np.arange(N) - I0
    return RHO0 + np.where(j <= 0, G1, G2) * j * dx


def activity_levels(dQ, M, nc, dx):
    """s on the left, at the kink and on the right, for flux slopes dQ_k/drho and maxima M_k:
    j_k = dQ_k (rho(x+1) - rho(x-1)) / 2 (Eqs. 28-29), s = (sum_k (j_k/M_k)^2 / nc)^(1/2) (Eqs. 30-31)."""
    K = math.sqrt(sum((q / m) ** 2 for q, m in zip(dQ, M)) / nc)
    return K * G1 * dx, K * 0.5 * (G1 + G2) * dx, K * G2 * dx


def test_sensor_a_filter_weights_at_a_slope_kink():
    # 1D, Sensor A: beta = beta_max - (beta_max - beta_min) clip(C s_bar) (Eq. 34) with s_bar the
    # (1/4, 1/2, 1/4) filter of the two-level activity.  Uniform 1/3 taps change s_bar at cells
    # I0-1 and I0+1 by about 10% of its value; no filter changes it by more.
    p = wl.SOD_1D.resized(N)
    dx = p.dx
    rho = density_kink(dx)
    W0 = wl.conserved(p.eos, rho, [np.full(N, U)], np.full(N, P0))
    s = O.OracleSolver.for_problem(p, threads=1, c_sensor=4.0)
    s.init(W0)
    beta = s.eval_beta()[0]
    rmax = rho.max()
    dQ = [U, U * U, 0.5 * U ** 3]
    M = [rmax * U, rmax * U * U + P0, (P0 / (GAM - 1.0) + 0.5 * rmax * U * U + P0) * U]
    sl, sk, sr = activity_levels(dQ, M, 3, dx)
    for i, sbar in kink_profile(sl, sk, sr).items():
        chi = 4.0 * sbar
        assert 0.0 < chi < 1.0
        expect = p.beta_max - (p.beta_max - p.beta_min) * chi
        assert abs(beta[i] - expect) <= 1e-14, (i, beta[i], expect)
    # the margin that other weights would miss by, in beta
    third = (2 * sl + sk) / 3.0
    assert abs((p.beta_max - p.beta_min) * 4.0 * (third - kink_profile(sl, sk, sr)[I0 - 1])) > 1e-4


def transpose_state(W):
    """The same state with x and y exchanged: (rho, rho u, rho v, rho E) -> transposed fields with
    the two momentum components swapped."""
    return np.ascontiguousarray(np.stack([W[0].T, W[2].T, W[1].T, W[3].T]))


@pytest.mark.parametrize("axis", ["x", "y"])
def test_activity_filter_at_a_density_kink_2d(axis):
    # 2D: density kink along x at velocity (U, 0) and constant P.  Q_x = (rho U, rho U^2 + P, 0,
    # (P/(gamma-1) + rho U^2/2 + P) U) is linear in rho, Q_y = (0, 0, P, 0) is uniform, so the
    # flux activity s is the 1D two-level profile with nc = 4 components and M_2 = P (from Q_y).
    # The state is uniform along y, so s_bar is the filter along x alone.  axis = "y" runs the
    # transposed state (filter along y).
    p = wl.QUADRANTS_2D.resized(N)
    dx = p.dx
    rho = np.tile(density_kink(dx), (N, 1))
    W0 = wl.conserved(p.eos, rho, [np.full_like(rho, U), np.zeros_like(rho)], np.full_like(rho, P0))
    if axis == "y":
        W0 = transpose_state(W0)
    s = O.OracleSolver.for_problem(p, threads=1)
    s.init(W0)
    F = s.sensor_fields()
    sbar = F["s_bar"] if axis == "x" else F["s_bar"].T
    sraw = F["s"] if axis == "x" else F["s"].T
    rmax = rho.max()
    dQ = [U, U * U, 0.0, 0.5 * U ** 3]
    M = [rmax * U, rmax * U * U + P0, P0, (P0 / (GAM - 1.0) + 0.5 * rmax * U * U + P0) * U]
    sl, sk, sr = activity_levels(dQ, M, 4, dx)
    np.testing.assert_allclose(sraw[:, 2:I0], sl, rtol=1e-13)
    np.testing.assert_allclose(sraw[:, I0], sk, rtol=1e-13)
    np.testing.assert_allclose(sraw[:, I0 + 1:N - 2], sr, rtol=1e-13)
    for i, v in kink_profile(sl, sk, sr).items():
        np.testing.assert_allclose(sbar[:, i], v, rtol=1e-13, err_msg=f"column {i}")
    # no dilatation (u = rho U / rho rounds to U within an ulp): theta ~ 0 (Eq. 33), so
    # beta = beta_max although s > 0 (Eq. 35)
    assert np.abs(F["theta"]).max() <= 1e-20
    np.testing.assert_allclose(F["beta"], p.beta_max, rtol=0, atol=1e-15)


@pytest.mark.parametrize("axis", ["x", "y"])
def test_ducros_ratio_and_its_filter_at_a_kink(axis):
    # Velocity in two straight pieces meeting at cell I0 (uniform along y, rho = 1, P = 1):
    #   i <= I0: u_x = a (x - x_I0), u_y = 0   (pure dilatation: dil = a, vort = 0)
    #   i >= I0: u_x = 0, u_y = b (x - x_I0)   (pure shear: dil = 0, vort = b)
    # Central differences of straight pieces are exact: at the kink dil = a/2, vort = b/2.  So
    # theta = a^2/(a^2 + eps) left, (a/2)^2/((a/2)^2 + (b/2)^2 + eps) at I0, exactly 0 right
    # (Eqs. 32-33, eps in the units of |grad u|^2), and theta_bar = S[theta] has the kink profile.
    # With no filter theta_bar(I0 + 1) would be 0; with 1/3 taps theta_k/3 instead of theta_k/4.
    # Then beta = beta_max - (beta_max - beta_min) clip(C s_bar theta_bar) (Eq. 35).
    a, b, eps = 1.0, 2.0, 1e-6
    p = wl.QUADRANTS_2D.resized(N)
    dx = p.dx
    xi = (np.arange(N) - I0) * dx
    ux = np.tile(np.where(xi <= 0, a * xi, 0.0), (N, 1))
    uy = np.tile(np.where(xi >= 0, b * xi, 0.0), (N, 1))
    one = np.ones((N, N))
    W0 = wl.conserved(p.eos, one, [ux, uy], one)
    if axis == "y":
        W0 = transpose_state(W0)
    s = O.OracleSolver.for_problem(p, threads=1, ducros_eps=eps)
    s.init(W0)
    F = s.sensor_fields()
    tr = (lambda A: A) if axis == "x" else (lambda A: A.T)
    theta, thbar, sbar, beta = tr(F["theta"]), tr(F["theta_bar"]), tr(F["s_bar"]), tr(F["beta"])
    tl = a * a / (a * a + eps)
    tk = 0.25 * a * a / (0.25 * a * a + 0.25 * b * b + eps)
    np.testing.assert_allclose(theta[:, 1:I0], tl, rtol=1e-14)
    np.testing.assert_allclose(theta[:, I0], tk, rtol=1e-14)
    assert np.array_equal(theta[:, I0 + 1:N - 1], np.zeros((N, N - 2 - I0)))
    expect = kink_profile(tl, tk, 0.0)
    for i, v in expect.items():
        np.testing.assert_allclose(thbar[:, i], v, rtol=1e-14, atol=1e-16, err_msg=f"column {i}")
    assert np.array_equal(thbar[:, I0 + 2:N - 1], np.zeros((N, N - 3 - I0)))
    # beta from the closed-form theta_bar and the filtered activity: the gate multiplies s_bar by
    # the filtered ratio, not by the raw one (at I0 + 1 the raw theta is 0 but beta < beta_max)
    assert sbar[0, I0 + 1] > 0.0
    for i, v in expect.items():
        chi = np.clip(p.c_sensor * sbar[:, i] * v, 0.0, 1.0)
        np.testing.assert_allclose(beta[:, i], p.beta_max - (p.beta_max - p.beta_min) * chi, rtol=0, atol=1e-15)
    assert (beta[:, I0 + 1] < p.beta_max).all()
