"""Domain totals (vlbm_get_totals) and checkpoint / resume (vlbm_save_state, vlbm_load_state).

* Totals: the compensated device sum equals the exactly rounded sum (math.fsum) of the field
  vlbm_get_W returns, and on periodic domains the step conserves them (Sec. III A): drift after
  100 steps <= 1e-13 of sum |W_k| in FP64; FP32 storage rounds every stored deviation, so its
  drift is bounded by a few FP32 unit roundoffs per step instead.
* Resume: a state saved after n steps and loaded into a fresh solver continues bit for bit like
  the saving solver (fields, time, link speed, history), for both precisions and both step forms,
  including a state saved right after vlbm_init; damaged or mismatched buffers are rejected.
"""
import dataclasses
import math

import numpy as np
import pytest

from paper_2609_10639_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def _vortex(n=96):
    prob = dataclasses.replace(wl.VORTEX_ADJOINT_2D.resized(n), extent=(0.0, 10.0, 0.0, 10.0))
    return prob, wl.vortex_density_2d(prob)


@pytest.mark.parametrize("precision", ["fp64", "fp32_store"])
def test_totals_compensated_and_conserved(precision):
    import torch

    from paper_2609_10639_b300 import vlbm

    prob, W0 = _vortex()
    s = vlbm.Solver.for_problem(prob, precision=precision)
    s.init(torch.from_numpy(W0).cuda())
    T0 = s.totals()
    W = s.W().cpu().numpy()
    scale = np.abs(W).reshape(W.shape[0], -1).sum(axis=1)
    exact = np.array([math.fsum(W[k].ravel()) for k in range(W.shape[0])])
    assert np.all(np.abs(T0 - exact) <= 1e-15 * scale), (T0, exact)
    steps = 100
    assert s.step(steps) == steps
    T1 = s.totals()
    W = s.W().cpu().numpy()
    exact = np.array([math.fsum(W[k].ravel()) for k in range(W.shape[0])])
    assert np.all(np.abs(T1 - exact) <= 1e-15 * scale), (T1, exact)
    drift = np.abs(T1 - T0) / scale
    # FP32 storage: per step, the FP32 relaxation and the rounding of every stored deviation
    # (|d_i| <= |W|) move each total by a few units of 2^-24 of sum |W_k| at most
    bar = 1e-13 if precision == "fp64" else steps * 8 * 2.0 ** -24
    assert np.all(drift <= bar), (drift, bar)


@pytest.mark.parametrize("precision,algorithm", [("fp64", "two_pass"), ("fp64", "lookahead"),
                                                 ("fp32_store", "two_pass"), ("fp32_store", "lookahead")])
@pytest.mark.parametrize("n_save", [0, 37])
@pytest.mark.parametrize("gas", ["ideal", "vdw"])
def test_save_load_resumes_bit_for_bit(precision, algorithm, n_save, gas):
    # the van der Waals FP32 look-ahead path keeps the pressure between the steps; a restored state
    # recomputes it
    import torch

    from paper_2609_10639_b300 import vlbm

    if gas == "ideal":
        prob = wl.QUADRANTS_2D.resized(90, 70)
        W0 = torch.from_numpy(wl.quadrants_2d(prob)).cuda()
    else:
        prob = wl.BZT_2D.resized(90, 70)
        W0 = torch.from_numpy(wl.bzt_interface_2d(prob)).cuda()
    a = vlbm.Solver.for_problem(prob, precision=precision, algorithm=algorithm)
    a.init(W0)
    if n_save:
        assert a.step(n_save) == n_save
    blob = a.save_state()
    assert a.step(45) == 45
    b = vlbm.Solver.for_problem(prob, precision=precision, algorithm=algorithm)
    b.load_state(blob)
    assert b.time()[1] == n_save
    assert b.step(45) == 45
    assert torch.equal(a.W(), b.W())
    assert a.time() == b.time()
    ha, hb = a.history(), b.history()
    assert np.array_equal(ha[0], hb[0]) and np.array_equal(ha[1], hb[1])
    assert torch.equal(a.populations(), b.populations())


def test_load_rejects_damaged_and_mismatched_states():
    import torch

    from paper_2609_10639_b300 import vlbm

    prob = wl.QUADRANTS_2D.resized(40, 30)
    a = vlbm.Solver.for_problem(prob)
    a.init(torch.from_numpy(wl.quadrants_2d(prob)).cuda())
    a.step(5)
    blob = bytearray(a.save_state())
    bad = bytearray(blob)
    bad[len(bad) // 2] ^= 0x10
    b = vlbm.Solver.for_problem(prob)
    with pytest.raises(vlbm.VLBMError) as e:
        b.load_state(bytes(bad))
    assert e.value.status == vlbm.E_CHECKSUM
    with pytest.raises(vlbm.VLBMError) as e:
        b.load_state(bytes(blob[:-8]))
    assert e.value.status == vlbm.E_INVAL
    for other in (vlbm.Solver.for_problem(wl.QUADRANTS_2D.resized(41, 30)),
                  vlbm.Solver.for_problem(prob, precision="fp32_store")):
        with pytest.raises(vlbm.VLBMError) as e:
            other.load_state(bytes(blob))
        assert e.value.status == vlbm.E_INVAL
    b.load_state(bytes(blob))
    assert b.time()[1] == 5


@pytest.mark.parametrize("eos", ["vdw", "vdw_cvt"])
def test_kept_pressure_is_bit_identical_to_the_eos_evaluation(eos):
    # FP32 storage with a non-ideal gas: the strip kernel's look-ahead stage keeps the pressure of
    # the next state for the next step (no second FP64 EOS evaluation); the tile kernel evaluates the
    # EOS in both places.  The same operations on the same W: the runs agree to rounding (the two
    # kernels may contract multiply-adds differently); a pressure taken from the wrong step or
    # cell would differ by the change of a step, about 1e-3.
    import torch

    from paper_2609_10639_b300 import vlbm

    prob = (wl.BZT_2D if eos == "vdw" else wl.BZT_CVT_2D).resized(200, 130)
    W0 = torch.from_numpy(wl.bzt_interface_2d(prob)).cuda()
    out = []
    for tiling in ("strip", "tile"):
        g = vlbm.Solver.for_problem(prob, precision="fp32_store", algorithm="lookahead", tiling=tiling)
        g.init(W0)
        assert g.step(70) == 70
        out.append(g.W().cpu().numpy())
    rel = np.abs(out[0] - out[1]).reshape(4, -1).sum(1) / np.abs(out[1]).reshape(4, -1).sum(1)
    print(f"{eos}: kept pressure (strips) against the EOS evaluation (tiles), relative L1 {rel}")
    assert rel[[0, 3]].max() <= 1e-6