"""The largest grid the library accepts, checked through a property that holds at any size.

A periodic field that repeats a 64 x 64 block is stepped exactly like that block on its own
periodic 64 x 64 domain: every cell sees the same neighbours, and the global maxima (link speed,
flux normalisation) are the same.  So the GPU run on 11584 x 11584 cells (181 x 181 copies, just
below the 134,217,727-cell limit of the 32-bit population offsets) must equal, in every block, the
oracle's run of the block: relative max-norm 1e-11 after 100 FP64 steps, as on small grids.  In
FP32 storage each block must equal the GPU's own FP32 run of the block (the reference state
W_ref is the same mean, up to its last bit).  The first grid beyond the limit is rejected.
"""
import dataclasses

import numpy as np
import pytest

from paper_2609_10639_b300 import workloads as wl

pytestmark = pytest.mark.gpu
B, REPS = 64, 181  # 64 * 181 = 11584


def block_problem():
    p = dataclasses.replace(wl.QUADRANTS_2D.resized(B), bc=wl.PER, name="quadrants_2d_periodic")
    W0 = wl.quadrants_2d(p, states=[[0.5313, 0.0, 0.0, 0.4], [1.0, 0.7276, 0.0, 1.0], [0.8, 0.0, 0.0, 1.0],
                                    [1.0, 0.0, 0.7276, 1.0]])
    return p, W0


def blockwise_rel_maxnorm(Wbig, Wblock):
    """max over components of max |big - tiled block| / max |block|, on the device."""
    import torch

    nc = Wblock.shape[0]
    big = Wbig.view(nc, REPS, B, REPS, B)
    blk = torch.as_tensor(Wblock, device=Wbig.device).view(nc, 1, B, 1, B)
    num = (big - blk).abs().amax(dim=(1, 2, 3, 4))
    den = blk.abs().amax(dim=(1, 2, 3, 4)).clamp_min(1e-300)
    return float((num / den).max())


@pytest.mark.parametrize("precision", ["fp64", "fp32_store"])
def test_largest_grid_steps_like_its_repeated_block(precision):
    import torch

    from oracle import oracle as O
    from paper_2609_10639_b300 import vlbm

    p, W0 = block_problem()
    if precision == "fp64":
        o = O.OracleSolver.for_problem(p)
        o.init(W0)
        assert o.step(100) == 100
        ref, tol = o.W(), 1e-11
    else:
        s = vlbm.Solver.for_problem(p, precision=precision)
        s.init(W0)
        assert s.step(100) == 100
        ref, tol = s.W().cpu().numpy(), 1e-6
        s.close()
    big = dataclasses.replace(p, nx=B * REPS, ny=B * REPS, extent=(0.0, REPS, 0.0, REPS))
    assert big.ncells <= (2 ** 31 - 1) // 16
    g = vlbm.Solver.for_problem(big, precision=precision)
    W0big = torch.as_tensor(W0, device="cuda").repeat(1, REPS, REPS)
    g.init(W0big)
    del W0big
    assert g.step(100) == 100
    err = blockwise_rel_maxnorm(g.W(), ref)
    g.close()
    torch.cuda.empty_cache()
    assert err <= tol, f"{precision}: {err:.3e}"


def test_first_grid_beyond_the_limit_is_rejected():
    from paper_2609_10639_b300 import vlbm

    p, _ = block_problem()
    with pytest.raises(vlbm.VLBMError):
        vlbm.Solver.for_problem(dataclasses.replace(p, nx=11586, ny=11586, extent=(0.0, 1.0, 0.0, 1.0)))
    ok = vlbm.Solver.for_problem(dataclasses.replace(p, nx=11585, ny=11585, extent=(0.0, 1.0, 0.0, 1.0)))
    ok.close()
