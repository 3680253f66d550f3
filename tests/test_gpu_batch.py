"""vlbm_run_batch: independent runs whose host copies overlap the steps of the neighbouring runs.

* Each run's W, step count and time equal those of the same run through vlbm_init, vlbm_step and
  vlbm_get_W, bit for bit, for any mix of pinned host, pageable host and device arrays.
* An end time stops each run as vlbm_step does.
* A run that turns non-physical ends the batch with its status; later runs leave their outputs
  untouched.
"""
import numpy as np
import pytest

from paper_2609_10639_b300 import workloads as wl

pytestmark = pytest.mark.gpu
PROB = wl.QUADRANTS_2D.resized(300, 257)


def inputs(n):
    # the seeded four-quadrant input, scaled (P and rho E scale with rho: the same flow) and mirrored
    # (momentum component negated): distinct physical inputs (other seeds' random quadrant states
    # turn non-physical within 20 steps)
    base = wl.quadrants_2d(PROB)

    def flip(W, axis):
        W = np.flip(W, axis=2 - axis).copy()
        W[1 + axis] *= -1.0
        return W

    out = [base, 1.1 * base, flip(base, 0), flip(base, 1), 0.9 * flip(flip(base, 0), 1)]
    return out[:n]


def sequential(prob, W0s, n_steps, t_end=0.0, **kw):
    import torch

    from paper_2609_10639_b300 import vlbm

    g = vlbm.Solver.for_problem(prob, **kw)
    out = []
    for W0 in W0s:
        g.init(torch.from_numpy(W0).cuda())
        done = g.step(n_steps, t_end)
        out.append((g.W().cpu().numpy(), done, g.time()[0]))
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32_store"])
def test_batch_equals_sequential_runs(precision):
    import torch

    from paper_2609_10639_b300 import vlbm

    W0s = inputs(5)
    ref = sequential(PROB, W0s, 45, precision=precision)
    # inputs: pinned, pageable, device, pinned, pageable; outputs: pinned, device, pageable, ...
    ins = [torch.from_numpy(W0s[0]).pin_memory(), W0s[1], torch.from_numpy(W0s[2]).cuda(),
           torch.from_numpy(W0s[3]).pin_memory(), W0s[4]]
    outs = [torch.empty(W0s[0].shape, dtype=torch.float64).pin_memory(),
            torch.empty(W0s[0].shape, dtype=torch.float64, device="cuda"),
            np.empty(W0s[0].shape), torch.empty(W0s[0].shape, dtype=torch.float64).pin_memory(),
            torch.empty(W0s[0].shape, dtype=torch.float64, device="cuda")]
    g = vlbm.Solver.for_problem(PROB, precision=precision)
    outs, done = g.run_batch(ins, 45, outs=outs)
    assert done == [45] * 5
    for k, (Wr, nr, _) in enumerate(ref):
        Wb = outs[k] if isinstance(outs[k], np.ndarray) else outs[k].cpu().numpy()
        np.testing.assert_array_equal(Wb, Wr, err_msg=f"run {k}")
    # the handle holds the last run's state
    assert g.time()[0] == ref[-1][2]
    np.testing.assert_array_equal(g.W().cpu().numpy(), ref[-1][0])


def test_batch_with_end_time_and_shared_buffers():
    import torch

    from paper_2609_10639_b300 import vlbm

    W0s = inputs(3)
    t_end = 0.02
    ref = sequential(PROB, W0s, 10 ** 6, t_end)
    pinned_in = [torch.from_numpy(w).pin_memory() for w in W0s]
    out = torch.empty(W0s[0].shape, dtype=torch.float64).pin_memory()
    g = vlbm.Solver.for_problem(PROB)
    # one output array for every run: the readbacks run in order on one stream
    _, done = g.run_batch(pinned_in, 10 ** 6, t_end, outs=[out] * 3)
    assert done == [r[1] for r in ref]
    assert g.time()[0] == t_end
    np.testing.assert_array_equal(out.numpy(), ref[-1][0])
    # the same input array for every run
    outs, done = g.run_batch([pinned_in[1]] * 3, 30)
    for o in outs:
        np.testing.assert_array_equal(o.cpu().numpy(), outs[0].cpu().numpy())


def test_batch_stops_at_a_nonphysical_run():
    import torch

    from paper_2609_10639_b300 import vlbm

    W0s = inputs(3)
    W0s[1] = W0s[1].copy()
    W0s[1][0, 10, 10] = -0.5
    outs = [torch.full(W0s[0].shape, 7.0, dtype=torch.float64).pin_memory() for _ in range(3)]
    g = vlbm.Solver.for_problem(PROB)
    with pytest.raises(vlbm.NonPhysicalState):
        g.run_batch([torch.from_numpy(w).pin_memory() for w in W0s], 20, outs=outs)
    np.testing.assert_array_equal(outs[0].numpy(), sequential(PROB, W0s[:1], 20)[0][0])
    assert (outs[2].numpy() == 7.0).all()


def test_batch_argument_checks():
    import torch

    from paper_2609_10639_b300 import vlbm

    g = vlbm.Solver.for_problem(PROB)
    W0 = torch.from_numpy(inputs(1)[0]).cuda()
    with pytest.raises(vlbm.VLBMError) as ei:
        g.run_batch([W0], -1)
    assert ei.value.status == vlbm.E_INVAL
    with pytest.raises(ValueError):
        g.run_batch([W0[:, :10]], 5)  # too few values
    with pytest.raises(ValueError):
        g.run_batch([W0], 5, outs=[])
    assert g.run_batch([], 5) == ([], [])


def test_batch_on_a_pinned_inflow_grid():
    # the pinned-inflow boundary: the batch needs the inflow state as vlbm_init does, and each run
    # equals its sequential counterpart
    import torch

    from paper_2609_10639_b300 import vlbm

    prob = wl.SHOCK_VORTEX_IDEAL.resized(120, 45)
    W0 = wl.shock_vortex_2d(prob)
    runs = [W0, W0 * 1.05]
    s = vlbm.Solver(vlbm.Config(dim=2, nx=prob.nx, ny=prob.ny, extent=prob.extent, bc=prob.bc, eos=prob.eos))
    with pytest.raises(vlbm.VLBMError) as ei:
        s.run_batch([torch.from_numpy(w).cuda() for w in runs], 10)
    assert ei.value.status == vlbm.E_STATE
    g = vlbm.Solver.for_problem(prob)
    outs, done = g.run_batch([torch.from_numpy(w).pin_memory() for w in runs], 40)
    assert done == [40, 40]
    ref = sequential(prob, runs, 40)
    for k in range(2):
        np.testing.assert_array_equal(outs[k].cpu().numpy(), ref[k][0])
