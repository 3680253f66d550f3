"""GPU adjoint (vlbm_adjoint through the C ABI) against the dual-number oracle and central finite
differences.

Objective J = sum_x g(x) rho(x, T).  The link-speed sequence is that of the forward run, held
fixed.  Dual numbers (forward mode, same non-smooth conventions) give <dJ/dW0, v> and dJ/dgamma
exactly up to rounding: bar 1e-9 relative.  Central differences (eps = 1e-6) of the GPU forward
run on the full 1024^2 / 1000-step vortex workload, 20 seeded directions and gamma: bar 1e-4
relative.
"""
import dataclasses
import json
import os

import numpy as np
import pytest

from paper_2609_10639_b300 import workloads as wl

pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def _weight(prob):
    X, Y = wl.cell_centres(prob)
    L = prob.extent[1] - prob.extent[0]
    return np.ascontiguousarray(1.0 + 0.5 * np.cos(2 * np.pi * X / L) * (np.cos(2 * np.pi * Y / max(L, 1e-9)) if prob.dim == 2 else 1.0))


def _untie(W0, seed):
    """Relative 1e-6 per-cell noise: a piecewise-constant field has exact ties in the maxima M_k,
    whose derivative is defined only through the tie-break, and two implementations whose values
    differ in the last bit can break such ties on different elements."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(W0 * (1.0 + 1e-6 * rng.standard_normal(W0.shape[1:])))


def _cases():
    vort = dataclasses.replace(wl.VORTEX_ADJOINT_2D.resized(48, 40), extent=(0.0, 10.0, 0.0, 10.0 * 40 / 48))
    quad = wl.QUADRANTS_2D.resized(40, 28)
    sod = wl.SOD_1D.resized(160)
    bzt = wl.BZT_2D.resized(32, 24)
    return {
        "vortex_periodic_48x40": (vort, wl.vortex_density_2d(vort), 24, 8, {}),
        "quadrants_zerograd_40x28": (quad, _untie(wl.quadrants_2d(quad, states=GOLD["laxliu_config12"]["states_NE_NW_SW_SE"]), 1),
                                     18, 5, {}),
        "sod_1d_160": (sod, _untie(wl.sod_1d(sod), 2), 40, 7, {}),
        "bzt_vdw_32x24": (bzt, wl.bzt_interface_2d(bzt), 12, 4, {}),
        "vortex_const_beta": (vort, wl.vortex_density_2d(vort), 16, 16, {"beta_mode": "const", "beta_const": 0.8}),
    }


def _dual_dJ(prob, W0, n, g, sched, v=None, deos=None, **over):
    from oracle import oracle as O

    params = dict(cfl=prob.cfl, beta_min=prob.beta_min, beta_max=prob.beta_max, c_sensor=prob.c_sensor,
                  ducros_eps=prob.ducros_eps)
    params.update(over)
    d = O.DualOracleSolver(prob.dim, prob.nx, prob.ny, prob.dx, prob.bc, prob.eos, deos=deos, **params)
    d.set_schedule(sched)
    d.init(W0, v)
    assert d.step(n) == n
    _, dW = d.W()
    return float(np.sum(g * dW[0]))


@pytest.mark.parametrize("tape", ["tape", "lean_tape", "recompute"])
@pytest.mark.parametrize("case", list(_cases()))
def test_adjoint_matches_dual_numbers(case, tape):
    # tape: every segment in a full slot; lean_tape: every segment in a lean slot (states and sensor
    # planes; the adjoint evaluates W, u, Q itself); recompute: no tape
    import torch

    from oracle import oracle as O
    from paper_2609_10639_b300 import vlbm

    prob, W0, n, K, over = _cases()[case]
    g = _weight(prob)
    dJ_dWT = np.zeros_like(W0)
    dJ_dWT[0] = g
    s = vlbm.Solver.for_problem(prob, **over)
    nseg = -(-n // K)
    lean, _ = _tape_slot_doubles(s, prob, K, n, "fp64")
    s.set_adjoint_tape({"tape": -1, "lean_tape": 8 * nseg * lean, "recompute": 0}[tape])
    dW0, deos = s.adjoint(torch.from_numpy(W0).cuda(), n, K, torch.from_numpy(dJ_dWT).cuda())
    assert s.adjoint_info()[1] == (0 if tape == "recompute" else n)
    dW0 = dW0.cpu().numpy()
    assert s.time()[1] == n
    # the oracle's own link-speed sequence of the same run
    o = O.OracleSolver.for_problem(prob, **over)
    o.init(W0)
    c0 = o.time()[2]
    o.step(n)
    sched = np.concatenate([[c0], o.history()[1]])
    rng = np.random.default_rng(7)
    for _ in range(3):
        v = rng.standard_normal(W0.shape) * np.abs(W0).mean(axis=(1, 2), keepdims=True)
        ref = _dual_dJ(prob, W0, n, g, sched, v=v, **over)
        got = float(np.sum(dW0 * v))
        scale = float(np.sum(np.abs(dW0 * v)))
        assert abs(got - ref) <= 1e-9 * max(abs(ref), 1e-3 * scale), (case, got, ref)
    key = "gamma" if prob.eos["kind"] == "ideal" else "a"
    idx = ("gamma", "a", "b", "R", "cv").index(key)
    ref = _dual_dJ(prob, W0, n, g, sched, deos={key: 1.0}, **over)
    assert abs(deos[idx] - ref) <= 1e-9 * max(abs(ref), 1e-12), (case, deos[idx], ref)
    if prob.eos["kind"] == "vdw":
        for key in ("b", "R", "cv"):
            ref = _dual_dJ(prob, W0, n, g, sched, deos={key: 1.0}, **over)
            j = ("gamma", "a", "b", "R", "cv").index(key)
            assert abs(deos[j] - ref) <= 1e-9 * max(abs(ref), 1e-12), (case, key, deos[j], ref)


def test_adjoint_vortex_1024_central_differences():
    # The adjoint workload: 1024^2 periodic vortex with a 1e-2 density perturbation, 1000 steps,
    # checkpoints every 32 steps; J = sum g rho(T) with the seeded smooth weight g.
    import torch

    from paper_2609_10639_b300 import vlbm

    prob = wl.VORTEX_ADJOINT_2D
    W0 = wl.vortex_density_2d(prob)
    g = wl.objective_weight(prob)
    n, K = prob.n_steps, 32
    W0d = torch.from_numpy(W0).cuda()
    dJ = torch.zeros_like(W0d)
    dJ[0] = torch.from_numpy(g).cuda()
    s = vlbm.Solver.for_problem(prob)
    dW0, deos = s.adjoint(W0d, n, K, dJ)
    # replay the recorded link speeds for the perturbed runs
    _, cs = s.history()
    s0 = vlbm.Solver.for_problem(prob)
    s0.init(W0d)
    c0 = s0.time()[2]
    sched = np.concatenate([[c0], cs])
    gd = torch.from_numpy(g).cuda()

    def rho_T(Win, gamma=1.4):
        eos = dict(prob.eos)
        eos["gamma"] = gamma
        r = vlbm.Solver.for_problem(dataclasses.replace(prob, eos=eos))
        r.set_schedule(sched)
        r.init(Win)
        assert r.step(n) == n
        return r.W()[0]

    # central differences of J = sum g rho(T), differenced per cell before the sum, on the 20
    # seeded smooth directions
    eps = 1e-6
    dirs = wl.directions(prob, count=20)
    for v in dirs:
        vd = torch.from_numpy(np.ascontiguousarray(v)).cuda()
        fd = float((gd * (rho_T(W0d + eps * vd) - rho_T(W0d - eps * vd))).sum()) / (2 * eps)
        ad = float((dW0 * vd).sum())
        assert abs(ad - fd) <= 1e-4 * abs(fd), (ad, fd)
    fdg = float((gd * (rho_T(W0d, 1.4 + eps) - rho_T(W0d, 1.4 - eps))).sum()) / (2 * eps)
    assert abs(deos[0] - fdg) <= 1e-4 * abs(fdg), (deos[0], fdg)
    # the same gradient with every segment recomputed from its checkpoint (the tape, which held
    # most or all of the run above, off)
    assert s.adjoint_info()[1] > n // 2
    s.set_adjoint_tape(0)
    dW0r, deosr = s.adjoint(W0d, n, K, dJ)
    assert s.adjoint_info()[1] == 0
    err = float((dW0r - dW0).abs().max() / dW0.abs().max())
    print(f"1024^2 adjoint, recomputed segments against the tape: {err:.2e}")
    assert err <= 1e-12
    assert abs(deosr[0] - deos[0]) <= 1e-12 * abs(deos[0])


def test_autograd_function_matches_adjoint():
    import torch

    from paper_2609_10639_b300 import autograd, vlbm

    prob, W0, n, K, _ = _cases()["vortex_periodic_48x40"]
    g = torch.from_numpy(_weight(prob)).cuda()
    cfg = vlbm.Config(dim=prob.dim, nx=prob.nx, ny=prob.ny, extent=prob.extent, bc=prob.bc, eos=prob.eos, cfl=prob.cfl)
    W = torch.from_numpy(W0).cuda().requires_grad_(True)
    gam = torch.tensor(1.4, dtype=torch.float64, device="cuda", requires_grad=True)
    WT = autograd.run(W, gam, cfg, n, K)
    J = (g * WT[0]).sum()
    J.backward()
    s = vlbm.Solver(cfg)
    dJ = torch.zeros_like(W)
    dJ[0] = g
    dW0, deos = s.adjoint(W.detach(), n, K, dJ)
    assert torch.allclose(W.grad, dW0, rtol=0, atol=1e-13 * float(dW0.abs().max()))
    assert abs(float(gam.grad) - deos[0]) <= 1e-12 * abs(deos[0])


def test_fp32_storage_adjoint_against_fp64_adjoint():
    # FP32-storage run: checkpoints and recomputed states in FP32 storage, adjoint evaluated in
    # FP64 at those states.  Its gradient equals the FP64 adjoint's to 1e-4 (finite differences
    # of the FP32-storage run itself would be dominated by FP32 rounding).
    import torch

    from paper_2609_10639_b300 import vlbm

    prob = dataclasses.replace(wl.VORTEX_ADJOINT_2D.resized(256), n_steps=200)
    W0 = torch.from_numpy(wl.vortex_density_2d(prob)).cuda()
    dJ = torch.zeros_like(W0)
    dJ[0] = torch.from_numpy(wl.objective_weight(prob)).cuda()
    a = vlbm.Solver.for_problem(prob, precision="fp64")
    ga, ea = a.adjoint(W0, prob.n_steps, 32, dJ)
    b = vlbm.Solver.for_problem(prob, precision="fp32_store")
    gb, eb = b.adjoint(W0, prob.n_steps, 32, dJ)
    for v in wl.directions(prob, count=3):
        vd = torch.from_numpy(np.ascontiguousarray(v)).cuda()
        da, db = float((ga * vd).sum()), float((gb * vd).sum())
        assert abs(da - db) <= 1e-4 * abs(da), (da, db)
    assert abs(ea[0] - eb[0]) <= 1e-4 * abs(ea[0]), (ea[0], eb[0])


def test_adjoint_vortex_128_twenty_directions():
    # 128^2 periodic vortex, 200 steps, checkpoints every 32 steps: <dJ/dW0, v> against the dual
    # numbers on the 20 seeded smooth directions, and dJ/dgamma.
    import torch

    from oracle import oracle as O
    from paper_2609_10639_b300 import vlbm

    prob = dataclasses.replace(wl.VORTEX_ADJOINT_2D.resized(128), n_steps=200)
    W0 = wl.vortex_density_2d(prob)
    g = wl.objective_weight(prob)
    n = prob.n_steps
    dJ = np.zeros_like(W0)
    dJ[0] = g
    s = vlbm.Solver.for_problem(prob)
    dW0, deos = s.adjoint(torch.from_numpy(W0).cuda(), n, 32, torch.from_numpy(dJ).cuda())
    dW0 = dW0.cpu().numpy()
    o = O.OracleSolver.for_problem(prob)
    o.init(W0)
    c0 = o.time()[2]
    o.step(n)
    sched = np.concatenate([[c0], o.history()[1]])
    for v in wl.directions(prob, count=20):
        ref = _dual_dJ(prob, W0, n, g, sched, v=v)
        got = float(np.sum(dW0 * v))
        assert abs(got - ref) <= 1e-9 * abs(ref), (got, ref)
    ref = _dual_dJ(prob, W0, n, g, sched, deos={"gamma": 1.0})
    assert abs(deos[0] - ref) <= 1e-9 * abs(ref), (deos[0], ref)


def _tape_slot_doubles(s, prob, K, n, precision):
    """Doubles of one lean and one full tape slot: the segment's states in storage precision, plus
    on FP64 column strips the 8 sensor planes (lean) or all 22 kept planes (full) per state."""
    plane = prob.nx * (prob.ny if prob.dim == 2 else 1)
    state_vals = 2 * prob.dim * 4 * plane
    state = state_vals if precision == "fp64" else (state_vals + 1) // 2
    segn = min(K, n)
    strips64 = precision == "fp64" and prob.dim == 2 and s.cfg.tiling != "tile"
    return segn * (state + (8 * plane if strips64 else 0)), segn * (state + (22 * plane if strips64 else 0))


def _expected_tape(cap_bytes, lean, full, nseg):
    """As many lean slots as fit, the last of them made full with the memory left over."""
    T = min(nseg, cap_bytes // (8 * lean))
    Tf = min(T, (cap_bytes // 8 - T * lean) // (full - lean)) if full > lean else 0
    return T, Tf


@pytest.mark.parametrize("precision,tiling", [("fp64", "strip"), ("fp64", "tile"), ("fp32_store", "strip")])
def test_adjoint_tape_gives_the_recomputed_gradient(precision, tiling):
    # the same run with the tape off, partly on (a limit of 2.5 full slots: on FP64 strips three
    # lean slots, the last made full) and on for the whole run: the same gradient (the taped
    # states and kept quantities are those the recomputation produces), the reported taped steps
    # and tape size, and a state that vlbm_step continues exactly as a plain run of the same steps
    import torch

    from paper_2609_10639_b300 import vlbm

    prob = dataclasses.replace(wl.VORTEX_ADJOINT_2D.resized(96, 80), extent=(0.0, 10.0, 0.0, 10.0 * 80 / 96))
    W0 = torch.from_numpy(wl.vortex_density_2d(prob)).cuda()
    dJ = torch.zeros_like(W0)
    dJ[0] = torch.from_numpy(_weight(prob)).cuda()
    n, K = 45, 8  # six segments, the last one of five steps
    steps = [8, 8, 8, 8, 8, 5]
    out = {}
    for mode in ("off", "two", "all"):
        s = vlbm.Solver.for_problem(prob, precision=precision, tiling=tiling)
        lean, full = _tape_slot_doubles(s, prob, K, n, precision)
        cap = {"off": 0, "two": int(2.5 * 8 * full), "all": -1}[mode]
        s.set_adjoint_tape(cap)
        dW0, deos = s.adjoint(W0, n, K, dJ)
        fwd_ms, taped, used = s.adjoint_info()
        T, Tf = {"off": (0, 0), "all": (6, 6)}.get(mode) or _expected_tape(cap, lean, full, 6)
        assert taped == sum(steps[6 - T:]), (mode, taped, T)
        assert used == 8 * ((T - Tf) * lean + Tf * full), (mode, used, T, Tf)
        assert fwd_ms > 0.0
        assert s.time()[1] == n
        s.step(7)  # continues the run's final state
        out[mode] = (dW0.cpu().numpy(), deos, s.W().cpu().numpy())
    plain = vlbm.Solver.for_problem(prob, precision=precision, tiling=tiling)
    plain.init(W0)
    plain.step(n + 7)
    Wp = plain.W().cpu().numpy()
    ref = out["off"]
    for mode in ("two", "all"):
        g, e, Wc = out[mode]
        err = float(np.abs(g - ref[0]).max() / np.abs(ref[0]).max())
        print(f"{precision}/{tiling}/{mode}: gradient rel max difference to the recomputation {err:.2e}")
        assert err <= 1e-13, (mode, err)
        np.testing.assert_allclose(e, ref[1], rtol=1e-13)
    for mode in ("off", "two", "all"):
        d = float(np.abs(out[mode][2] - Wp).max() / np.abs(Wp).max())
        print(f"{precision}/{tiling}/{mode}: state 7 steps after the adjoint against a plain run: {d:.2e}")
        # FP64 and the untaped FP32 run: the same kernels and decisions.  Taped FP32 segments are
        # stepped in the two-pass form, the plain FP32 run in the look-ahead form (equal up to the
        # rounding of the FP32 moments)
        assert d <= (0.0 if precision == "fp64" or mode == "off" else 1e-6), (mode, d)
