"""The shock-vortex interaction (Sec. IV H) on the GPU: the pinned-inflow boundary through every
step-kernel form, against the oracle, and the full runs against the independent reference solver.

* FP64, 100 steps, the full grids (ideal gas 800 x 300, BZT van der Waals 1200 x 450), column
  strips and tiles, two-pass and look-ahead forms: relative max-norm of W against the oracle
  within the parity bar (1e-11, or ten times the oracle's own rounding spread where the flow
  amplifies rounding more).
* beta(x) of the state (vlbm_get_beta, the tile kernel's readback) against the oracle's.
* FP32 storage against FP64 after the same steps.
* The runs to t = 7 (ideal) and t = 15 (BZT) against the unsplit MUSCL-Rusanov reference at the
  same resolution and boundaries: the printed relative L1 density differences (0.093%, 0.114%)
  met within a factor 3/2.
"""
import dataclasses
import json
import os

import numpy as np
import pytest

from paper_2609_10639_b300 import workloads as wl

pytestmark = pytest.mark.gpu
TOL = 1e-11
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))
PROBS = {"ideal": wl.SHOCK_VORTEX_IDEAL, "bzt": wl.SHOCK_VORTEX_BZT}
# Runs past the first few hundred steps take beta_max = 0.99 (the start-up pulses of the initial
# discontinuity are not damped at beta = 1) and, for the BZT gas, beta_min = 0.6: the largest
# constant beta that carries that case to its end time (0.75, the other cases' value, turns it
# non-physical near t = 9.4, as the vortex core, compressed by the shock, nears the critical point).
LONG = {"ideal": dict(beta_max=0.99), "bzt": dict(beta_max=0.99, beta_min=0.6)}
_oracle_cache = {}


def rel_maxnorm(a, b):
    num = np.abs(a - b).reshape(a.shape[0], -1).max(axis=1)
    den = np.maximum(np.abs(b).reshape(b.shape[0], -1).max(axis=1), 1e-300)
    return float((num / den).max())


def oracle_run(name, steps):
    """The oracle's W after `steps` steps, its link-speed history, and its rounding spread (the
    same run from an input perturbed at 1e-16)."""
    key = (name, steps)
    if key not in _oracle_cache:
        from oracle import oracle as O

        prob = PROBS[name]
        W0 = wl.shock_vortex_2d(prob)
        o = O.OracleSolver.for_problem(prob)
        o.init(W0)
        o.step(steps)
        rng = np.random.default_rng(99)
        o2 = O.OracleSolver.for_problem(prob)
        o2.init(W0 * (1.0 + 1e-16 * rng.standard_normal(W0.shape)))
        o2.step(steps)
        _oracle_cache[key] = (o.W(), o.history()[1], rel_maxnorm(o2.W(), o.W()), o)
    return _oracle_cache[key]


@pytest.mark.parametrize("algorithm", ["two_pass", "lookahead"])
@pytest.mark.parametrize("tiling", ["strip", "tile"])
@pytest.mark.parametrize("name", ["ideal", "bzt"])
def test_shock_vortex_fp64_parity_100_steps(name, tiling, algorithm):
    import torch

    from paper_2609_10639_b300 import vlbm

    prob = PROBS[name]
    g = vlbm.Solver.for_problem(prob, algorithm=algorithm, tiling=tiling)
    g.init(torch.from_numpy(wl.shock_vortex_2d(prob)).cuda())
    assert g.step(100) == 100
    Wo, co, spread, _ = oracle_run(name, 100)
    bar = max(TOL, 10.0 * spread)
    err = rel_maxnorm(g.W().cpu().numpy(), Wo)
    print(f"{name}/{tiling}/{algorithm}: rel max-norm {err:.3e} (bar {bar:.1e}, oracle spread {spread:.1e})")
    assert err <= bar
    np.testing.assert_allclose(g.history()[1], co, rtol=max(1e-12, bar))


@pytest.mark.parametrize("name", ["ideal", "bzt"])
def test_shock_vortex_beta_field(name):
    import torch

    from paper_2609_10639_b300 import vlbm

    prob = PROBS[name]
    g = vlbm.Solver.for_problem(prob)
    g.init(torch.from_numpy(wl.shock_vortex_2d(prob)).cuda())
    g.step(100)
    _, _, spread, o = oracle_run(name, 100)
    bo = o.eval_beta()
    assert np.abs(g.beta() - bo).max() <= max(TOL, 10.0 * spread)
    assert bo.min() < 0.999  # the sensor acts at the (weak, M_s = 1.2) shock


@pytest.mark.parametrize("name", ["ideal", "bzt"])
def test_shock_vortex_fp32_storage_against_fp64(name):
    import torch

    from paper_2609_10639_b300 import vlbm

    prob = dataclasses.replace(PROBS[name], **LONG[name])
    W0 = torch.from_numpy(wl.shock_vortex_2d(prob)).cuda()
    out = {}
    for prec in ("fp64", "fp32_store"):
        g = vlbm.Solver.for_problem(prob, precision=prec)
        g.init(W0)
        assert g.step(500) == 500
        out[prec] = (g.W().cpu().numpy(), g.time()[0])
    (W64, t64), (W32, t32) = out["fp64"], out["fp32_store"]
    assert abs(t32 - t64) <= 1e-5 * t64
    rel = np.abs(W32 - W64).reshape(4, -1).sum(1) / np.abs(W64).reshape(4, -1).sum(1)
    print(f"{name}: FP32 storage vs FP64 after 500 steps, relative L1 per component {rel}")
    assert rel.max() <= 1e-4
    # the shock stays in the same cell in every row: argmax of |d rho/dx| past the vortex region
    gx64 = np.abs(np.diff(W64[0], axis=1))[:, 250:]
    gx32 = np.abs(np.diff(W32[0], axis=1))[:, 250:]
    assert np.abs(gx64.argmax(axis=1) - gx32.argmax(axis=1)).max() <= 1


REF_L1 = {"ideal": 0.00093, "bzt": 0.00114}  # Sec. IV H, relative L1 density against the reference


@pytest.mark.parametrize("name", ["ideal", "bzt"])
def test_shock_vortex_full_run_against_reference(name):
    import torch

    from oracle import oracle as O
    from paper_2609_10639_b300 import vlbm

    prob = dataclasses.replace(PROBS[name], **LONG[name])
    W0 = wl.shock_vortex_2d(prob)
    g = vlbm.Solver.for_problem(prob)
    g.init(torch.from_numpy(W0).cuda())
    g.step(10 ** 6, prob.t_end)
    assert g.time()[0] == prob.t_end
    Wg = g.W().cpu().numpy()
    Wr, _ = O.muscl_2d(prob.eos, W0, prob.dx, prob.t_end, bc=prob.bc, W_in=wl.inflow_state(prob))
    rel = float(np.abs(Wg[0] - Wr[0]).sum() / np.abs(Wr[0]).sum())
    print(f"{name}: relative L1(rho) against the reference {rel:.3e} (printed {REF_L1[name]:.2e})")
    assert rel <= 1.5 * REF_L1[name]


def test_pinned_inflow_needs_its_state_and_has_no_adjoint():
    import torch

    from paper_2609_10639_b300 import vlbm

    prob = wl.SHOCK_VORTEX_IDEAL.resized(64, 24)
    W0 = torch.from_numpy(wl.shock_vortex_2d(prob)).cuda()
    s = vlbm.Solver(vlbm.Config(dim=2, nx=prob.nx, ny=prob.ny, extent=prob.extent, bc=prob.bc, eos=prob.eos))
    with pytest.raises(vlbm.VLBMError) as ei:
        s.init(W0)
    assert ei.value.status == vlbm.E_STATE
    s.set_inflow(wl.inflow_state(prob))
    s.init(W0)
    assert s.step(5) == 5
    with pytest.raises(vlbm.VLBMError) as ei:
        s.adjoint(W0, 4, 2, torch.zeros_like(W0))
    assert ei.value.status == vlbm.E_UNSUPPORTED


@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (5, 1), (1, 7), (131, 57)])
@pytest.mark.parametrize("tiling", ["strip", "tile"])
def test_pinned_inflow_on_degenerate_and_ragged_grids(shape, tiling):
    # tiny and ragged grids with a pinned-inflow x-lo side: every cell next to the ghost column,
    # strips narrower than the halo, a single row, against the oracle after 25 steps (FP64, both forms)
    import torch

    from oracle import oracle as O
    from paper_2609_10639_b300 import vlbm

    nx, ny = shape
    prob = wl.Problem("inflow_small", 2, nx, ny, (0.0, 1.0, 0.0, ny / nx), wl.INFLOW_BC, wl.IDEAL14, 0.5, 0.0, 0)
    X, Y = wl.cell_centres(prob)
    rho = 1.0 + 0.2 * np.cos(2 * np.pi * Y) + 0.1 * X
    W0 = wl.conserved(prob.eos, rho, [1.1 + 0 * X, 0.1 * np.sin(2 * np.pi * Y)], 1.0 + 0.1 * X)
    W_in = wl.conserved(prob.eos, np.array(0.9), [np.array(1.3), np.array(0.0)], np.array(1.2)).reshape(-1)
    for algorithm in ("two_pass", "lookahead"):
        g = vlbm.Solver.for_problem(prob, algorithm=algorithm, tiling=tiling)
        g.set_inflow(W_in)
        g.init(torch.from_numpy(W0).cuda())
        assert g.step(25) == 25
        o = O.OracleSolver.for_problem(prob, threads=1)
        o.set_inflow(W_in)
        o.init(W0)
        o.step(25)
        Wg, Wo = g.W().cpu().numpy(), o.W()
        # per component, relative to its magnitude, or to 1e-3 of the state's where a component is
        # at rounding level (one column fed by the pinned state: rho v ~ 1e-16 after 25 steps)
        scale = np.maximum(np.abs(Wo).reshape(4, -1).max(1), 1e-3 * np.abs(Wo).max())
        err = float((np.abs(Wg - Wo).reshape(4, -1).max(1) / scale).max())
        assert err <= TOL, (shape, tiling, algorithm, err)
