"""Pins of the independent reference solver (oracle/muscl_reference.cpp) against what the
mathematics fixes, before it is used to check the 1D benchmarks of Secs. IV B-IV D.

* Sod problem: convergence to the exact Riemann solution (oracle/riemann_exact.py, two
  independent root finders) at the rate a second-order shock-capturing scheme reaches on a
  solution with a shock and a contact (between 0.5 and 1 in L1), with no new extrema.
* Smooth contact wave: a density wave advected at constant u and P is an exact solution of the
  Euler equations for any equation of state, so the ideal-gas and van der Waals runs are
  compared with the shifted initial profile; second order in L1 (minmod clips the extrema, so a
  little below 2).  A wrong EOS inversion e(rho, P) leaves P non-uniform and fails this.
* Periodic domain: mass, momentum and energy conserved to rounding.
"""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import riemann_exact as RX
from paper_2609_10639_b300 import workloads as wl

VDW = {"kind": "vdw", "a": 3.0, "b": 1.0 / 3.0, "R": 1.0, "cv": 80.0}


def test_muscl_sod_converges_to_exact_solution():
    l1 = []
    for n in (200, 400, 800):
        p = wl.SOD_1D.resized(n)
        W, steps = O.muscl_1d(p.eos, wl.sod_1d(p)[:, 0, :], p.dx, "zerograd", 0.2)
        assert steps > 0
        X, _ = wl.cell_centres(p)
        rho_e, u_e, p_e = RX.solution(X.ravel(), 0.2, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4)
        l1.append(p.dx * np.abs(W[0] - rho_e).sum())
        # no new extrema: density within the two initial states, velocity not negative
        assert W[0].min() >= 0.125 - 1e-12 and W[0].max() <= 1.0 + 1e-12
        assert (W[1] / W[0]).min() >= -1e-12
    orders = np.log2(np.array(l1[:-1]) / np.array(l1[1:]))
    assert l1[-1] < 2.5e-3
    assert np.all(orders > 0.6) and np.all(orders < 1.2), (l1, orders)


@pytest.mark.parametrize("eos", [wl.IDEAL14, VDW], ids=["ideal", "vdw"])
def test_muscl_second_order_on_a_smooth_contact_wave(eos):
    rho0 = 0.6 if eos["kind"] == "vdw" else 1.0  # van der Waals: a dense single-phase state
    P0 = 1.2 if eos["kind"] == "vdw" else 1.0
    errs = []
    for n in (64, 128, 256):
        x = (np.arange(n) + 0.5) / n
        rho = rho0 * (1.0 + 0.2 * np.sin(2 * np.pi * x))
        W0 = wl.conserved(eos, rho, [np.full(n, 1.0)], np.full(n, P0))
        W, _ = O.muscl_1d(eos, W0, 1.0 / n, "periodic", 1.0)  # one period: back to the start
        errs.append(np.abs(W[0] - rho).sum() / n)
        u = W[1] / W[0]
        assert np.abs(u - 1.0).max() < 20 * errs[-1] + 1e-12  # u stays uniform to the error level
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.7), (errs, orders)


def test_muscl_conserves_on_a_periodic_domain():
    n = 300
    x = (np.arange(n) + 0.5) / n
    rho = np.where(np.abs(x - 0.5) < 0.2, 1.0, 0.3) + 0.1 * np.sin(6 * np.pi * x)
    W0 = wl.conserved(wl.IDEAL14, rho, [0.3 * np.cos(2 * np.pi * x)], 0.5 + 0.4 * (x > 0.3))
    W, steps = O.muscl_1d(wl.IDEAL14, W0, 1.0 / n, "periodic", 0.3)
    assert steps > 50
    tot0, tot = W0.sum(axis=1), W.sum(axis=1)
    assert np.all(np.abs(tot - tot0) <= 1e-13 * np.abs(W0).sum(axis=1))


def test_muscl_reports_a_non_physical_state():
    n = 50
    W0 = wl.conserved(wl.IDEAL14, np.ones(n), [np.zeros(n)], np.ones(n))
    W0[0, 10] = -1.0
    with pytest.raises(ValueError):
        O.muscl_1d(wl.IDEAL14, W0, 1.0 / n, "zerograd", 0.1)


def test_muscl_2d_planar_problems_and_transpose():
    # A Sod problem along x on a 200 x 4 grid stays uniform across (every row identical, the y
    # fluxes cancel exactly), matches the exact solution like the 1D method, and the same problem
    # along y is its exact transpose (u and v exchanged): the two face directions share no
    # index arithmetic, so a transposed operand or a wrong stride fails this.
    n = 200
    x = (np.arange(n) + 0.5) / n
    rho, P = np.where(x < 0.5, 1.0, 0.125), np.where(x < 0.5, 1.0, 0.1)
    z = np.zeros((4, n))
    Wx = wl.conserved(wl.IDEAL14, np.tile(rho, (4, 1)), [z, z], np.tile(P, (4, 1)))
    Wy = wl.conserved(wl.IDEAL14, np.tile(rho, (4, 1)).T.copy(), [z.T, z.T], np.tile(P, (4, 1)).T.copy())
    A, _ = O.muscl_2d(wl.IDEAL14, Wx, 1.0 / n, 0.2)
    B, _ = O.muscl_2d(wl.IDEAL14, Wy, 1.0 / n, 0.2)
    assert all(np.array_equal(A[:, 0], A[:, j]) for j in range(1, 4))
    assert np.array_equal(A, B.transpose(0, 2, 1)[[0, 2, 1, 3]])
    rho_e, _, _ = RX.solution(x, 0.2, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4)
    assert np.abs(A[0, 0] - rho_e).mean() < 6e-3


def test_muscl_2d_second_order_on_an_advected_bump():
    # a smooth density bump carried diagonally at constant (u, v) and P (an exact solution for
    # any EOS) stays away from the boundaries; minmod clips its peak, so the L1 order is ~1.55
    errs = []
    bump = lambda X, Y: 1.0 + 0.2 * np.exp(-((X - 0.35) ** 2 + (Y - 0.35) ** 2) / 0.01)
    for n in (64, 128, 256):
        x = (np.arange(n) + 0.5) / n
        X, Y = np.meshgrid(x, x, indexing="xy")
        W0 = wl.conserved(wl.IDEAL14, bump(X, Y), [np.full_like(X, 0.5), np.full_like(X, 0.5)], np.ones_like(X))
        W, _ = O.muscl_2d(wl.IDEAL14, W0, 1.0 / n, 0.3)
        errs.append(np.abs(W[0] - bump(X - 0.15, Y - 0.15)).mean())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.45), (errs, orders)
