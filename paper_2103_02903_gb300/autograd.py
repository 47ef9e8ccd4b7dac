"""torch.autograd binding of the adjoint (mr_lbm_adjoint).

``trajectory_functional(conserved0, s, cfg, nsteps, ...)`` returns the
functional J of the adaptive trajectory started from the conserved moments
``conserved0`` (CUDA tensor [ncons, N_J], float64) with relaxation rates
``s`` (tensor [16]); backward gives dJ/d conserved0 and dJ/d s from the
library's adjoint kernels (mesh frozen per step, checkpoints every
``checkpoint_every`` steps).  Marshalling only: the forward and the
gradients are computed by mr_lbm_adjoint in one call.
"""
from __future__ import annotations

import torch

from .binding import Solver


class TrajectoryFunctional(torch.autograd.Function):
    @staticmethod
    def forward(ctx, conserved0, s, cfg, nsteps, checkpoint_every, functional):
        c = dict(cfg)
        c["s"] = [float(v) for v in s.detach().to("cpu", torch.float64)]
        solver = Solver(c)
        u = conserved0.detach().contiguous()
        J, g_u, g_s = solver.adjoint(u, nsteps, checkpoint_every, functional)
        solver.close()
        ctx.save_for_backward(g_u, torch.as_tensor(g_s, dtype=s.dtype, device=s.device))
        return torch.tensor(J, dtype=torch.float64, device=conserved0.device)

    @staticmethod
    def backward(ctx, gJ):
        g_u, g_s = ctx.saved_tensors
        return gJ * g_u, gJ.to(g_s.device) * g_s, None, None, None, None


def trajectory_functional(conserved0, s, cfg, nsteps, checkpoint_every=100, functional="ke_sum"):
    return TrajectoryFunctional.apply(conserved0, s, cfg, nsteps, checkpoint_every, functional)
