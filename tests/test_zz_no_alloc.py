"""The allocation-free entry point vlbm_beta_noalloc, called through the C ABI.

It serves callers that cannot allocate device memory (a host application that owns all device
memory through its own pool, code running while a CUDA graph is captured, a fixed-budget loop):
all its scratch lives in a static device array inside the library.  Its output must equal what
the handle-based vlbm_get_beta returns for the same state, on consecutive calls (the array is
shared and keeps the previous call's contents), and grids beyond the array's capacity must be
refused.  This file is collected last so that a run stopping at the first failure has already run
every other test; it also passes when run alone in a fresh process.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))
TOL = 1e-11  # the FP64 parity bar of the other GPU tests


def _cases():
    from paper_2609_10639_b300 import workloads as wl

    quad = wl.QUADRANTS_2D.resized(257, 131)  # ragged: several 32 x 16 tiles plus partial ones
    return [
        (quad, wl.quadrants_2d(quad, states=GOLD["laxliu_config12"]["states_NE_NW_SW_SE"])),
        (wl.SOD_1D, wl.sod_1d(wl.SOD_1D)),
    ]


@pytest.mark.parametrize("which", [0, 1], ids=["2d_257x131", "1d_1000"])
def test_beta_noalloc_matches_handle_on_consecutive_calls(which):
    import torch

    from paper_2609_10639_b300 import vlbm

    prob, W0 = _cases()[which]
    s = vlbm.Solver.for_problem(prob)
    s.init(torch.from_numpy(W0).cuda())
    for steps in (7, 13):  # two calls in a row, on two different states
        s.step(steps)
        ref = s.beta()
        # the state in the library's storage layout [i][y][x][4] (components last, padded to 4)
        fi = s.populations()  # interface layout [i][k][y][x]
        f = torch.zeros((s.q, s.ny, s.nx, 4), dtype=torch.float64, device="cuda")
        f[..., : s.nc] = fi.permute(0, 2, 3, 1)
        out = torch.full((s.ny, s.nx), float("nan"), dtype=torch.float64, device="cuda")
        vlbm.beta_noalloc(s.cfg, f, out, in_place=True)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= TOL
        assert ref.min() < 1.0  # the sensor is active on these states


@pytest.mark.parametrize("dim", [1, 2])
def test_beta_noalloc_pulls_post_collision_populations(dim):
    # in_place = 0: the caller's buffer holds post-collision populations f*, which the call pulls
    # across the links, f_i(x) = f*_i(x - sigma_i) (Eq. 21).  On a periodic grid f* is the state
    # rolled by +sigma_i, so the result must equal the handle's beta of the state itself.
    import dataclasses

    import torch

    from paper_2609_10639_b300 import vlbm, workloads as wl

    if dim == 2:
        prob = dataclasses.replace(wl.QUADRANTS_2D.resized(200, 97), bc=wl.PER)
        W0 = wl.quadrants_2d(prob, states=GOLD["laxliu_config12"]["states_NE_NW_SW_SE"])
    else:
        prob = dataclasses.replace(wl.SOD_1D.resized(600), bc=wl.PER)
        W0 = wl.sod_1d(prob)
    s = vlbm.Solver.for_problem(prob)
    s.init(torch.from_numpy(W0).cuda())
    for steps in (9, 4):  # two calls in a row, on two different states
        s.step(steps)
        ref = s.beta()
        fi = s.populations()  # [i][k][y][x]
        # sigma_i in the lattice order {x-, x+, y-, y+}: f*_i(x) = f_i(x + sigma_i)
        rolls = [(1, 3), (-1, 3), (1, 2), (-1, 2)]
        fstar = torch.stack([torch.roll(fi[i], shifts=rolls[i][0], dims=rolls[i][1] - 1) for i in range(s.q)])
        f = torch.zeros((s.q, s.ny, s.nx, 4), dtype=torch.float64, device="cuda")
        f[..., : s.nc] = fstar.permute(0, 2, 3, 1)
        out = torch.full((s.ny, s.nx), float("nan"), dtype=torch.float64, device="cuda")
        vlbm.beta_noalloc(s.cfg, f, out, in_place=False)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= TOL
        assert ref.min() < 1.0


def test_beta_noalloc_rejects_grids_beyond_its_scratch():
    import torch

    from paper_2609_10639_b300 import vlbm

    cfg = vlbm.Config(dim=2, nx=2048, ny=1025)  # 2,099,200 cells > 2,097,152
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(vlbm.VLBMError) as ei:
        vlbm.beta_noalloc(cfg, f, out)
    assert ei.value.status == vlbm.E_INVAL
    # axes whose product wraps around in 64-bit arithmetic are refused too
    for nx, ny in ((2 ** 32, 2 ** 32), (2 ** 21 + 1, 1), (1, 2 ** 40)):
        with pytest.raises(vlbm.VLBMError) as ei:
            vlbm.beta_noalloc(vlbm.Config(dim=2, nx=nx, ny=ny), f, out)
        assert ei.value.status == vlbm.E_INVAL
