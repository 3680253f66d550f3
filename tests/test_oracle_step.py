"""Pins of the oracle's lattice, equilibrium, reprojection and full step (Sec. III) against
invariants, closed forms and independent reference updates.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2609_10639_b300 import workloads as wl

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))
SIG = {1: np.array([[-1.0], [1.0]]), 2: np.array([[-1.0, 0.0], [1.0, 0.0], [0.0, -1.0], [0.0, 1.0]])}


def random_state(rng, dim, eos):
    """A random hyperbolic state (c_s^2 > 0, Eq. 14) as a conserved vector."""
    while True:
        if eos["kind"] == "ideal":
            rho, P = rng.uniform(0.05, 5.0), rng.uniform(0.01, 10.0)
        else:
            rho, P = rng.uniform(0.3, 0.9), rng.uniform(0.8, 1.3)
        if O.eos_eval(eos, rho, wl.internal_energy(eos, rho, P))[1] > 0:
            break
    vel = rng.uniform(-2.0, 2.0, dim)
    return wl.conserved(eos, np.array(rho), list(vel), np.array(P)).ravel()


# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("eos", [wl.IDEAL14, wl.VDW_REDUCED], ids=["ideal", "vdw"])
def test_equilibrium_consistency(dim, eos):
    # Eq. (19): sum_i f_i^eq = W and sum_i c_i f_i^eq = Q(W), for random states and link speeds.
    rng = np.random.default_rng(1 + dim)
    for _ in range(2000):
        W = random_state(rng, dim, eos)
        c = rng.uniform(0.5, 50.0)
        fe = O.feq(dim, eos, c, W)
        Qf = O.flux(dim, eos, W)
        np.testing.assert_allclose(fe.sum(axis=0), W, rtol=4e-15, atol=4e-15 * np.abs(W).max())
        mom = (c * SIG[dim]).T @ fe  # (dim, NC)
        # a few ulp of the largest term c |f_i|, which cancels in the difference
        np.testing.assert_allclose(mom, Qf, rtol=1e-14, atol=4e-16 * c * np.abs(fe).max())


def normal_shock_ideal(gam, M, rho1=1.0, P1=1.0):
    """Textbook stationary normal shock of an ideal gas (Rankine-Hugoniot)."""
    c1 = math.sqrt(gam * P1 / rho1)
    u1 = M * c1
    rho2 = rho1 * (gam + 1) * M * M / ((gam - 1) * M * M + 2)
    P2 = P1 * (1 + 2 * gam / (gam + 1) * (M * M - 1))
    return (rho1, u1, P1), (rho2, u1 * rho1 / rho2, P2)


@pytest.mark.parametrize("dim", [1, 2])
def test_flux_continuous_across_ideal_normal_shock(dim):
    # A stationary shock carries equal flux Q_x on both sides (Eqs. 9-10): a dropped pressure
    # term or a wrong energy flux breaks this.  Cross-checked with the printed state (Sec. IV H).
    g = GOLD["ideal_normal_shock"]
    (r1, u1, P1), (r2, u2, P2) = normal_shock_ideal(g["gamma"], g["Ms"])
    for x, ref in [(u1, g["u1"]), (r2, g["rho2"]), (u2, g["u2"]), (P2, g["P2"])]:
        assert abs(x - ref) <= 1e-3
    eos = {"kind": "ideal", "gamma": g["gamma"]}
    vel1 = [u1] + [0.3] * (dim - 1)  # tangential velocity is continuous too
    vel2 = [u2] + [0.3] * (dim - 1)
    W1 = wl.conserved(eos, np.array(r1), vel1, np.array(P1)).ravel()
    W2 = wl.conserved(eos, np.array(r2), vel2, np.array(P2)).ravel()
    np.testing.assert_allclose(O.flux(dim, eos, W1)[0], O.flux(dim, eos, W2)[0], rtol=1e-13)


def test_flux_continuous_across_bzt_normal_shock():
    # The BZT stationary shock printed in Sec. IV H (3-digit states): flux equal to ~1e-3.
    g = GOLD["bzt_normal_shock"]
    e = GOLD["bzt_vdw_eos"]
    eos = {"kind": "vdw", "a": e["a"], "b": e["b"], "R": e["R"], "cv": e["R"] / (e["gamma"] - 1)}
    u1 = g["Ms"] * g["cs1"]
    W1 = wl.conserved(eos, np.array(g["rho1"]), [u1], np.array(g["P1"])).ravel()
    W2 = wl.conserved(eos, np.array(g["rho2"]), [g["u2"]], np.array(g["P2"])).ravel()
    Q1, Q2 = O.flux(1, eos, W1)[0], O.flux(1, eos, W2)[0]
    assert np.all(np.abs(Q1 - Q2) / np.abs(Q1) < 6e-3)


# --------------------------------------------------------------------------------------------
def moments(dim, c, f):
    """W, J_alpha (Eq. 38) and K (Eq. 39) of one cell's populations f[i][k]."""
    ci = c * SIG[dim]
    W = f.sum(axis=0)
    J = ci.T @ f
    K = ((ci[:, 0] ** 2 - ci[:, 1] ** 2) @ f) if dim == 2 else None
    return W, J, K


@pytest.mark.parametrize("dim", [1, 2])
def test_reprojection_invariants(dim):
    rng = np.random.default_rng(7)
    for _ in range(500):
        f = rng.normal(size=(2 * dim, dim + 2))
        c0, c1 = rng.uniform(0.5, 20), rng.uniform(0.5, 20)
        g = O.reproject(dim, c0, c1, f)
        W0, J0, K0 = moments(dim, c0, f)
        W1, J1, K1 = moments(dim, c1, g)
        np.testing.assert_allclose(W1, W0, atol=1e-13)
        np.testing.assert_allclose(J1, J0, rtol=1e-12, atol=1e-12 * max(1, np.abs(J0).max()))
        if dim == 2:
            np.testing.assert_allclose(K1, K0, rtol=1e-12, atol=1e-12 * max(1, np.abs(K0).max()))
        back = O.reproject(dim, c1, c0, g)
        np.testing.assert_allclose(back, f, atol=1e-13 * max(1.0, c0 / c1, c1 / c0) ** 2)


@pytest.mark.parametrize("dim", [1, 2])
def test_reprojection_of_equilibrium_is_equilibrium(dim):
    # With K = 0 and J = Q(W), Eq. (40) reduces to Eq. (20) at the new link speed.
    rng = np.random.default_rng(9)
    for _ in range(200):
        W = random_state(rng, dim, wl.IDEAL14)
        c0, c1 = rng.uniform(1, 20), rng.uniform(1, 20)
        g = O.reproject(dim, c0, c1, O.feq(dim, wl.IDEAL14, c0, W))
        np.testing.assert_allclose(g, O.feq(dim, wl.IDEAL14, c1, W), rtol=1e-13, atol=1e-13 * np.abs(W).max())


# --------------------------------------------------------------------------------------------
def _flux_np(dim, eos, W):
    """Eq. (10) in numpy for whole fields (ideal gas only), for the reference updates below."""
    g = eos["gamma"]
    rho = W[0]
    u = [W[1 + a] / rho for a in range(dim)]
    E = W[-1]
    P = (g - 1.0) * (E - 0.5 * rho * sum(x * x for x in u))
    out = []
    for a in range(dim):
        q = [W[1 + a]] + [W[1 + b] * u[a] + (P if a == b else 0.0) for b in range(dim)] + [(E + P) * u[a]]
        out.append(np.stack(q))
    cs = np.sqrt(g * P / rho)
    smax = max(float((np.abs(u[a]) + cs).max()) for a in range(dim))
    return out, smax


def _shift(a, d, axis, bc):
    """a at index j + d along axis with the boundary rule (periodic wrap or edge clamp)."""
    n = a.shape[axis]
    idx = np.arange(n) + d
    idx = idx % n if bc == "periodic" else np.clip(idx, 0, n - 1)
    return np.take(a, idx, axis=axis)


@pytest.mark.parametrize("dim,bc", [(1, "zerograd"), (1, "periodic"), (2, "zerograd"), (2, "periodic")])
def test_half_beta_step_is_lax_friedrichs(dim, bc):
    # beta = 1/2 makes the post-collision populations the equilibrium (Eq. 22), so one step is the
    # Lax-Friedrichs update (Sec. III B): W_new = mean of the 2D neighbours of W minus
    # sum_alpha (Q_alpha(x + e_alpha) - Q_alpha(x - e_alpha)) / (2c), with c = s_max / CFL.
    p = wl.quadrants_2d if dim == 2 else wl.sod_1d
    prob = (wl.QUADRANTS_2D.resized(24, 17) if dim == 2 else wl.SOD_1D.resized(40))
    prob = type(prob)(**{**prob.__dict__, "bc": (bc,) * 4})
    W0 = p(prob)
    s = O.OracleSolver.for_problem(prob, beta_mode="const", beta_const=0.5)
    s.init(W0)
    W = s.W()
    s.step(1)
    Qs, smax = _flux_np(dim, prob.eos, W)
    c = smax / prob.cfl
    ref = np.zeros_like(W)
    for a in range(dim):
        ax = 2 - a  # x is the last axis
        ref += (_shift(W, -1, ax, bc) + _shift(W, 1, ax, bc)) / (2 * dim)
        ref -= (_shift(Qs[a], 1, ax, bc) - _shift(Qs[a], -1, ax, bc)) / (2 * c)
    np.testing.assert_allclose(s.W(), ref, rtol=1e-13, atol=1e-13 * np.abs(W).max())


def test_uniform_state_is_a_fixed_point():
    for dim in (1, 2):
        prob = wl.QUADRANTS_2D.resized(12, 9) if dim == 2 else wl.SOD_1D.resized(16)
        W0 = np.zeros((dim + 2, prob.ny, prob.nx))
        W0[:] = wl.conserved(prob.eos, np.array(1.3), [0.4] * dim, np.array(0.9)).reshape(-1, 1, 1)
        s = O.OracleSolver.for_problem(prob)
        s.init(W0)
        s.step(300)
        np.testing.assert_allclose(s.W(), W0, rtol=1e-13)
        assert np.all(s.beta() == 1.0)


@pytest.mark.parametrize("eos", [wl.IDEAL14, wl.VDW_REDUCED], ids=["ideal", "vdw"])
@pytest.mark.parametrize("beta_mode", ["sensor", "const"])
def test_conservation_on_periodic_domain(eos, beta_mode):
    # Discrete conservation of mass, momentum and energy for any beta and EOS (Sec. III A).
    prob = wl.Problem("per", 2, 32, 24, (0, 1, 0, 24 / 32), wl.PER, eos, 0.5, 0.0, 100)
    X, Y = wl.cell_centres(prob)
    if eos["kind"] == "ideal":
        rho = 1 + 0.5 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y / 0.75)
        P = 1 + 0.3 * np.cos(2 * np.pi * X)
    else:
        rho = 0.7 + 0.05 * np.sin(2 * np.pi * X)
        P = 1.0 + 0.02 * np.cos(2 * np.pi * Y / 0.75)
    W0 = wl.conserved(eos, rho, [0.3 * np.sin(2 * np.pi * Y / 0.75), 0.2 + 0 * X], P)
    s = O.OracleSolver.for_problem(prob, beta_mode=beta_mode, beta_const=0.8)
    s.init(W0)
    S0 = [math.fsum(s.W()[k].ravel()) for k in range(4)]
    s.step(100)
    S1 = [math.fsum(s.W()[k].ravel()) for k in range(4)]
    scale = [math.fsum(np.abs(W0[k]).ravel()) for k in range(4)]
    for a, b, sc in zip(S0, S1, scale):
        assert abs(a - b) <= 1e-13 * sc


def test_beta_one_is_non_dissipative_and_beta_half_is_lax_friedrichs_damping():
    # Linear acoustic wave on a periodic line at a fixed link speed.  beta = 1 keeps the mode
    # amplitude (Sec. III B: |z| = 1); beta = 1/2 damps it by the Lax-Friedrichs factor
    # |z|^2 = cos^2(k dx) + (c_s / c)^2 sin^2(k dx) per step.
    n, amp, gam = 64, 1e-6, 1.4
    prob = wl.Problem("ac", 1, n, 1, (0, 1, 0, 0), wl.PER, {"kind": "ideal", "gamma": gam}, 0.5, 0.0, 0)
    X, _ = wl.cell_centres(prob)
    cs0 = math.sqrt(gam)
    k = 2 * np.pi * 2
    rho = 1 + amp * np.cos(k * X)
    u = amp * cs0 * np.cos(k * X)  # right-running simple wave
    P = 1 + amp * cs0 ** 2 * np.cos(k * X)
    W0 = wl.conserved(prob.eos, rho, [u], P)
    c = cs0 / 0.5
    steps = 128
    res = {}
    for beta in (1.0, 0.5):
        s = O.OracleSolver.for_problem(prob, beta_mode="const", beta_const=beta)
        s.set_schedule(np.full(steps + 1, c))
        s.init(W0)
        s.step(steps)
        d = s.W()[0, 0] - 1.0
        res[beta] = 2 * abs(np.fft.rfft(d)[2]) / n / amp
    assert abs(res[1.0] - 1.0) < 2e-3
    th = k * prob.dx
    z = math.sqrt(math.cos(th) ** 2 + (cs0 / c) ** 2 * math.sin(th) ** 2)
    assert res[0.5] == pytest.approx(z ** steps, rel=1e-3)
    assert res[0.5] < 0.5


def test_transpose_symmetry():
    # Swapping x and y (and u and v) commutes with the 2D step (Lax-Liu configuration 12 states).
    prob = wl.QUADRANTS_2D.resized(20, 20)
    W0 = wl.quadrants_2d(prob, states=GOLD["laxliu_config12"]["states_NE_NW_SW_SE"])
    WT = np.ascontiguousarray(np.stack([W0[0].T, W0[2].T, W0[1].T, W0[3].T]))
    a = O.OracleSolver.for_problem(prob)
    b = O.OracleSolver.for_problem(prob)
    a.init(W0)
    b.init(WT)
    a.step(30)
    b.step(30)
    Wa, Wb = a.W(), b.W()
    Wb_back = np.stack([Wb[0].T, Wb[2].T, Wb[1].T, Wb[3].T])
    np.testing.assert_allclose(Wa, Wb_back, rtol=1e-12, atol=1e-12)


def test_mirror_symmetry_1d():
    # Reflecting x -> -x (and u -> -u) commutes with the 1D step, including the sensor.
    prob = wl.SOD_1D.resized(50)
    W0 = wl.sod_1d(prob)
    WM = np.ascontiguousarray(np.stack([W0[0][:, ::-1], -W0[1][:, ::-1], W0[2][:, ::-1]]))
    a = O.OracleSolver.for_problem(prob)
    b = O.OracleSolver.for_problem(prob)
    a.init(W0)
    b.init(WM)
    a.step(40)
    b.step(40)
    Wb = b.W()
    np.testing.assert_allclose(a.W(), np.stack([Wb[0][:, ::-1], -Wb[1][:, ::-1], Wb[2][:, ::-1]]), rtol=1e-12, atol=1e-12)


def test_scaling_invariance():
    # W -> lambda W leaves u, e, c_s (ideal gas), the normalised sensor (Eq. 30) and hence beta
    # and the link speed unchanged, so the whole evolution scales by lambda.
    prob = wl.QUADRANTS_2D.resized(18, 14)
    W0 = wl.quadrants_2d(prob, states=GOLD["laxliu_config12"]["states_NE_NW_SW_SE"])
    lam = 3.7
    a = O.OracleSolver.for_problem(prob)
    b = O.OracleSolver.for_problem(prob)
    a.init(W0)
    b.init(lam * W0)
    a.step(25)
    b.step(25)
    np.testing.assert_allclose(b.W(), lam * a.W(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(b.beta(), a.beta(), atol=1e-12)


def test_final_step_lands_on_t_end_and_history():
    prob = wl.SOD_1D.resized(100)
    s = O.OracleSolver.for_problem(prob)
    s.init(wl.sod_1d(prob))
    n = s.step(10 ** 6, 0.05)
    t, nn, c = s.time()
    assert t == 0.05 and nn == n
    dt, cc = s.history()
    assert len(dt) == n and math.fsum(dt) == pytest.approx(0.05, rel=1e-14)
    np.testing.assert_allclose(dt, prob.dx / cc, rtol=1e-15)
    # the replayed schedule reproduces the run
    r = O.OracleSolver.for_problem(prob)
    W0 = wl.sod_1d(prob)
    s0 = O.OracleSolver.for_problem(prob)
    s0.init(W0)
    c0 = s0.time()[2]
    r.set_schedule(np.concatenate([[c0], cc]))
    r.init(W0)
    r.step(n)
    np.testing.assert_array_equal(r.W(), s.W())


def test_nonphysical_state_is_rejected():
    prob = wl.SOD_1D.resized(16)
    W0 = wl.sod_1d(prob)
    W0[0, 0, 3] = -1.0
    s = O.OracleSolver.for_problem(prob)
    with pytest.raises(ValueError):
        s.init(W0)


# --------------------------------------------------------------------------------------------
# Shock sensor (Sec. III D, Eqs. 28-35) on states where its chain has a closed form.
@pytest.mark.parametrize("g,c_sensor,clipped", [(0.5, 4.0, False), (40.0, 4.0, False), (0.5, 200.0, False), (0.5, 1000.0, True)])
def test_sensor_a_closed_form_on_a_density_ramp(g, c_sensor, clipped):
    # rho = rho0 + g x at constant u = U, P = P0 (ideal gas): every flux component is linear in
    # rho (Q_0 = rho U, Q_1 = rho U^2 + P0, Q_2 = (P0/(gamma-1) + rho U^2/2 + P0) U), so the
    # central jump j_k = dx g dQ_k/drho (U, U^2, U^3/2) is exact and the same in every interior
    # cell, M_k = |Q_k| of the densest cell, s = sqrt(sum_k (j_k/M_k)^2 / 3) is constant, the
    # normalised box filter leaves it unchanged away from the two edge cells, and
    # beta = beta_max - (beta_max - beta_min) clip(C s, 0, 1).  A missing 1/2 in the jump, a local
    # instead of global M_k, an unnormalised filter or a reversed map fails this.
    n, rho0, U, P0, gam = 64, 1.0, 0.8, 1.5, 1.4
    p = wl.SOD_1D.resized(n)
    x = (np.arange(n) + 0.5) / n
    rho = rho0 + g * x
    W0 = wl.conserved(p.eos, rho, [np.full(n, U)], np.full(n, P0))
    s = O.OracleSolver.for_problem(p, threads=1, c_sensor=c_sensor)
    s.init(W0)
    beta = s.eval_beta()[0]
    dx, rmax = p.dx, rho.max()
    j = dx * g * np.array([U, U * U, 0.5 * U ** 3])
    M = np.array([rmax * U, rmax * U * U + P0, (P0 / (gam - 1.0) + 0.5 * rmax * U * U + P0) * U])
    s_val = math.sqrt(np.sum((j / M) ** 2) / 3.0)
    chi = min(max(c_sensor * s_val, 0.0), 1.0)
    assert (chi == 1.0) == clipped
    expect = p.beta_max - (p.beta_max - p.beta_min) * chi
    assert np.abs(beta[2:-2] - expect).max() <= 1e-13


def test_sensor_b_is_gated_by_the_ducros_ratio():
    # 2D: the same ramp along x (uniform in y, velocity along x constant) has no dilatation and no
    # vorticity, so theta = 0 (Eq. 33) and beta = beta_max everywhere, although the flux activity
    # alone would lower it; a pure shear v = V x (vorticity, no dilatation) also gives theta = 0.
    n = 32
    p = wl.QUADRANTS_2D.resized(n)
    X, Y = wl.cell_centres(p)
    for vel in ([np.full_like(X, 0.8), np.zeros_like(X)], [np.zeros_like(X), 0.3 * X]):
        W0 = wl.conserved(p.eos, 1.0 + 40.0 * X, vel, np.full_like(X, 1.5))
        s = O.OracleSolver.for_problem(p, threads=1)
        s.init(W0)
        assert np.array_equal(s.eval_beta(), np.full((n, n), p.beta_max))
