"""Terminal-velocity mismatch as a differentiable PyTorch function.

``TerminalVelocityLoss.apply(drag_scale, diameter, u0, problem)`` runs the
coupled solver forward through the C ABI (``lbm_adj_forward``) and, on
``backward``, the hand-written adjoint kernels (``lbm_adj_backward``).  Inputs:
the drag scale s_D (scalar tensor), the bubble diameter d (scalar tensor, the
same for every bubble of the problem) and the initial liquid velocity field u0
(tensor [3, nz, ny, nx]); output: L = (ubar - target)^2 with ubar the mean rise
velocity over the last ``window`` steps.  Gradients flow to all three inputs,
so any parametrisation of them built from torch operations is differentiated
by autograd around the adjoint.
"""
from dataclasses import dataclass, field

import numpy as np
import torch

from . import lbm


@dataclass
class TerminalVelocityProblem:
    dims: tuple
    omega: float
    positions: np.ndarray            # [n, 3] bubble centres at release
    steps: int
    checkpoint_every: int
    window: int
    target: float
    walls: int = lbm.LBM_WALL_ALL
    g: float = 1e-5
    params: dict = field(default_factory=dict)

    def column(self, drag_scale, diameter, u0):
        p = lbm.lbm_default_params()
        p.g = self.g
        p.drag_scale = float(drag_scale)
        for k, v in self.params.items():
            setattr(p, k, v)
        col = lbm.Column(self.dims, self.omega, self.walls, params=p)
        lbm.lbm_set_fields(col.ctx, None, np.ascontiguousarray(u0, dtype=np.float64).reshape(-1))
        n = len(self.positions)
        lbm.lbm_set_bubbles(col.ctx, np.asarray(self.positions, dtype=np.float64).reshape(-1),
                            np.zeros(3 * n), np.full(n, float(diameter)))
        return col

    def loss(self, drag_scale, diameter, u0):
        return TerminalVelocityLoss.apply(drag_scale, diameter, u0, self)


class TerminalVelocityLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, drag_scale, diameter, u0, problem):
        col = problem.column(drag_scale.item(), diameter.item(), u0.detach().cpu().numpy())
        loss = lbm.lbm_adj_forward(col.ctx, problem.steps, problem.checkpoint_every,
                                   problem.window, problem.target)
        ctx.col = col
        ctx.shape = u0.shape
        ctx.device = u0.device
        return torch.tensor(loss, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        g_sd, g_d, g_u0 = lbm.lbm_adj_backward(ctx.col.ctx, float(grad_out), want_u0=True)
        ctx.col.close()
        grad_u0 = torch.from_numpy(g_u0.reshape(ctx.shape)).to(ctx.device)
        return (torch.tensor(g_sd, dtype=torch.float64), torch.tensor(float(np.sum(g_d)),
                dtype=torch.float64), grad_u0, None)
