"""Differentiation through the CUDA forward model (torch.autograd).

``FwiFunction`` wraps ``fwi_model`` (forward traces) and ``fwi_adjoint`` (the adjoint
wavefield with the fused cross-correlation) so that a misfit written with ordinary torch
operations on the traces back-propagates to the contrasts of the chosen parameterization.

Backward calls ``fwi_adjoint`` with the incoming trace-space gradient as its residual; the
library re-runs the forward with wavefield history and, when the whole history does not fit
the workspace budget, keeps checkpoints of (p, vx, vz) and recomputes each segment before
its adjoint (``fwi_workspace_bytes`` plans it).  The gradient of the other parameterizations
is available from ``fwi_adjoint`` directly; autograd returns the pair that parameterizes the
input.
"""
from __future__ import annotations

import torch

from . import fwi


class FwiFunction(torch.autograd.Function):
    """traces = F(xi_a, xi_b) for fixed grid, parameterization and acquisition."""

    # library kernels launched by the most recent backward (autograd may run the backward on
    # its own thread, where the library's per-thread launch counter lives)
    last_backward_launches = 0

    @staticmethod
    def forward(ctx, xi_a, xi_b, grid, pz, src_xy, wavelet, rec_xy, budget_bytes):
        traces = fwi.fwi_model(grid, pz, xi_a.detach(), xi_b.detach(), src_xy, wavelet, rec_xy)
        ctx.save_for_backward(xi_a.detach(), xi_b.detach(), src_xy, wavelet, rec_xy)
        ctx.grid, ctx.pz, ctx.budget = grid, pz, budget_bytes
        return traces

    @staticmethod
    def backward(ctx, grad_traces):
        xi_a, xi_b, src_xy, wavelet, rec_xy = ctx.saved_tensors
        g = ctx.grid
        ns, nr = src_xy.reshape(-1, 2).shape[0], rec_xy.reshape(-1, 2).shape[0]
        work = fwi.workspace(g, ns, nr, fwi.OP_ADJOINT, ctx.budget)
        G = fwi.fwi_adjoint(g, ctx.pz, xi_a, xi_b, src_xy, wavelet, rec_xy,
                            grad_traces.contiguous().float(), work=work)
        FwiFunction.last_backward_launches = fwi.launch_count()
        ga = G[ctx.pz, 0].to(xi_a.dtype) if ctx.needs_input_grad[0] else None
        gb = G[ctx.pz, 1].to(xi_b.dtype) if ctx.needs_input_grad[1] else None
        return ga, gb, None, None, None, None, None, None


def model(xi_a, xi_b, grid, pz, src_xy, wavelet, rec_xy, budget_bytes=None):
    """Differentiable forward modelling: traces [ns][nr][nt] (float32, CUDA)."""
    return FwiFunction.apply(xi_a, xi_b, grid, pz, src_xy, wavelet, rec_xy, budget_bytes)
