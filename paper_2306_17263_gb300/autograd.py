"""torch.autograd binding of the forward run and its reverse pass.

``propagate_ez(grid, ez0, nsteps)`` returns E_z after ``nsteps`` steps of the compact scheme
from E_z^0 = ez0 with H^{1/2} from the Taylor series of Sec. 5.1 (ms_taylor_init).  Its
backward is ms_adjoint_run: the exact transpose of that linear map, applied on the GPU.
Both directions run in the library's CUDA kernels; torch only holds the device memory.
"""
from __future__ import annotations

import torch

from . import Grid


def _grid_sync_in(grid: Grid):
    # work queued by torch on its stream must finish before the grid's stream reads it
    torch.cuda.current_stream().synchronize()


class PropagateEz(torch.autograd.Function):
    @staticmethod
    def forward(ctx, ez0: torch.Tensor, grid: Grid, nsteps: int):
        ez0 = ez0.detach().to(torch.float64).contiguous()
        _grid_sync_in(grid)
        grid.taylor_init_device(ez0)
        grid.run(nsteps)
        ez, hx, hy = (torch.empty(s, dtype=torch.float64, device=ez0.device) for s in grid.shapes())
        grid.get_fields_device(ez, hx, hy)
        grid.sync()
        ctx.grid, ctx.nsteps = grid, int(nsteps)
        return ez

    @staticmethod
    def backward(ctx, grad_ez: torch.Tensor):
        g = grad_ez.detach().to(torch.float64).contiguous()
        out = torch.empty_like(g)
        _grid_sync_in(ctx.grid)
        ctx.grid.adjoint_run_device(ctx.nsteps, g, out)
        ctx.grid.sync()
        return out, None, None


def propagate_ez(grid: Grid, ez0: torch.Tensor, nsteps: int) -> torch.Tensor:
    """E_z^{nsteps} from E_z^0 = ez0 (differentiable with respect to ez0)."""
    return PropagateEz.apply(ez0, grid, nsteps)
