"""torch.autograd.Function over the objective calls of libsophie.

ProbeObjective maps the eps_r values of a box of design cells to
J = dt * sum_{n=1..N} (probe value after step n)^2 of a run of N steps from
zero fields. Its forward sets the materials (the background with the design
box replaced), resets the grid and records the objective
(sophie_objective_forward); its backward runs the reverse sweep
(sophie_objective_grad_eps). Both run in libsophie's kernels; this module only
moves arrays.
"""

from __future__ import annotations

import numpy as np
import torch

from . import sophie as so


class ProbeObjective(torch.autograd.Function):
    """J(eps_design); eps_design has shape (nk, nj, ni) (x fastest)."""

    @staticmethod
    def forward(ctx, eps_design: torch.Tensor, grid: so.Grid, eps_background: np.ndarray,
                sigma: np.ndarray, box: tuple, probe: tuple, nsteps: int, checkpoint_every: int = 50):
        i0, j0, k0, ni, nj, nk = box
        eps = np.array(eps_background, dtype=np.float32, copy=True)
        eps[k0:k0 + nk, j0:j0 + nj, i0:i0 + ni] = eps_design.detach().to("cpu", torch.float32).numpy()
        grid.set_materials(eps, sigma)
        grid.reset()
        grid.objective_set_design(*box)  # the backward's box: traces instead of recomputation
        J = grid.objective_forward(nsteps, *probe, checkpoint_every)
        ctx.grid, ctx.box = grid, box
        ctx.dtype, ctx.device = eps_design.dtype, eps_design.device
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_J: torch.Tensor):
        g = ctx.grid.objective_grad_eps(*ctx.box)
        grad = torch.from_numpy(g) * grad_J.to("cpu", torch.float64)
        return (grad.to(ctx.device, ctx.dtype),) + (None,) * 7


def probe_objective(eps_design, grid, eps_background, sigma, box, probe, nsteps, checkpoint_every=50):
    return ProbeObjective.apply(eps_design, grid, eps_background, sigma, box, probe, nsteps, checkpoint_every)
