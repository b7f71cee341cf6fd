"""torch.autograd.Function for the time-averaged mean-pressure shift (argument marshalling only:
the forward run, the checkpointed recomputation and the reverse sweep run in the CUDA library,
lb_pressure_shift_gradient)."""
from __future__ import annotations

from dataclasses import replace

import torch

from . import LatticeParams, Simulation


class MeanPressureShift(torch.autograd.Function):
    """L(G, lambda_s, lambda_d) = <Pbar>_T(kT) - <Pbar>_T(kT = 0) on one lattice, fixed noise.

    Usage: ``MeanPressureShift.apply(G, lambda_s, lambda_d, base, steps, ckpt_every, precision,
    options)`` with 0-d tensors for the three parameters, a LatticeParams ``base`` for the rest and
    optionally a dict of Simulation options of the step (``astar``, ``wall_fixed``,
    ``noise_loc``).  The reverse sweep runs when the function is applied; backward scales the
    stored gradient."""

    @staticmethod
    def forward(ctx, G, lambda_s, lambda_d, base: LatticeParams, steps: int, ckpt_every: int = 100,
                precision: str = "fp64", options: dict | None = None):
        lam_e = base.lambda_s if base.lambda_e is None else base.lambda_e  # held fixed
        p = replace(base, G=float(G), lambda_s=float(lambda_s), lambda_d=float(lambda_d), lambda_e=lam_e)
        with Simulation(p, precision=precision, **(options or {})) as sim:
            loss, grad = sim.pressure_shift_gradient(steps, ckpt_every)
        ctx.save_for_backward(torch.as_tensor(grad, dtype=torch.float64))
        return torch.tensor(loss, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gout):
        (g,) = ctx.saved_tensors
        return gout * g[0], gout * g[1], gout * g[2], None, None, None, None, None
