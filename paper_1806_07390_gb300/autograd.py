"""torch.autograd binding of the library's boundary-outflow objective and its adjoint.

`boundary_outflow(grid, base_state, rho0, kappa0, dt, nsteps, k)` returns the radiation energy J
that leaves through the upper x boundary in nsteps steps, starting from `base_state` with its
density replaced by rho0 (pressure, velocity and radiation held fixed) and opacity normalisation
kappa0.  Gradients with respect to rho0 and kappa0 come from the hand-written adjoint kernels
(fx_adjoint_forward stores a checkpoint every k steps; fx_adjoint_backward recomputes each
segment and runs the stage adjoints backwards).  This module only marshals arguments.
"""
from __future__ import annotations

import torch


class BoundaryOutflow(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho0, kappa0, grid, base_state, dt, nsteps, k):
        grid.upload(base_state)
        grid.set_density(rho0.detach().contiguous())
        k0 = float(kappa0)
        grid.set_kappa0(k0)
        ws = grid.adjoint_workspace(nsteps, k)
        J = grid.adjoint_forward(ws, dt, nsteps, k)
        ctx.grid, ctx.ws, ctx.args = grid, ws, (float(dt), int(nsteps), int(k), k0)
        ctx.rho_dtype, ctx.k_dtype = rho0.dtype, kappa0.dtype
        return torch.tensor(J, dtype=torch.float64, device=rho0.device)

    @staticmethod
    def backward(ctx, gJ):
        dt, nsteps, k, k0 = ctx.args
        ctx.grid.set_kappa0(k0)
        _, grho, dk = ctx.grid.adjoint_backward(ctx.ws, dt, nsteps, k, seed=float(gJ))
        gk = torch.tensor(dk, dtype=ctx.k_dtype, device=grho.device)
        return grho.to(ctx.rho_dtype), gk, None, None, None, None, None


def boundary_outflow(grid, base_state, rho0: torch.Tensor, kappa0: torch.Tensor, dt: float,
                     nsteps: int, k: int) -> torch.Tensor:
    return BoundaryOutflow.apply(rho0, kappa0, grid, base_state, dt, nsteps, k)
