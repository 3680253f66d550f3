"""torch.autograd.Function over the VLBM run: W(T) = run(W0, EOS parameter) with the hand-written
adjoint of the library (vlbm_adjoint) as its backward.  Every step runs in the CUDA library."""
from __future__ import annotations

import dataclasses

import torch

from . import vlbm

EOS_KEYS = ("gamma", "a", "b", "R", "cv")


class VLBMFunction(torch.autograd.Function):
    """forward(W0, eos_param, cfg, n_steps, checkpoint_every, param_name) -> W(T).

    W0: CUDA float64 tensor (D+2, ny, nx); eos_param: 0-d float64 tensor holding the EOS parameter
    `param_name` (e.g. "gamma"), which overrides cfg.eos[param_name].  backward returns dJ/dW0 and
    dJ/d(eos_param); the link-speed sequence of the forward run is held fixed."""

    @staticmethod
    def forward(ctx, W0, eos_param, cfg: vlbm.Config, n_steps: int, checkpoint_every: int, param_name: str = "gamma"):
        eos = dict(cfg.eos)
        eos[param_name] = float(eos_param)
        cfg = dataclasses.replace(cfg, eos=eos)
        W0c = W0.detach().contiguous()
        s = vlbm.Solver(cfg)
        s.init(W0c)
        done = s.step(n_steps)
        if done != n_steps:
            raise RuntimeError(f"run stopped after {done} of {n_steps} steps")
        WT = s.W()
        ctx.solver, ctx.n_steps, ctx.K, ctx.param = s, n_steps, checkpoint_every, param_name
        ctx.save_for_backward(W0c)
        return WT

    @staticmethod
    def backward(ctx, grad_WT):
        (W0,) = ctx.saved_tensors
        dW0, deos = ctx.solver.adjoint(W0, ctx.n_steps, ctx.K, grad_WT.detach().to(torch.float64).contiguous())
        g = torch.tensor(deos[EOS_KEYS.index(ctx.param)], dtype=torch.float64, device=W0.device)
        return dW0, g, None, None, None, None


def run(W0, eos_param, cfg: vlbm.Config, n_steps: int, checkpoint_every: int = 32, param_name: str = "gamma"):
    return VLBMFunction.apply(W0, eos_param, cfg, n_steps, checkpoint_every, param_name)
