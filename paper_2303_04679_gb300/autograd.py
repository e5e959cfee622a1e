"""torch.autograd.Function over the library's hand-written adjoint.

The forward pass evaluates the mODIL loss of caller-owned level values on the
GPU (modil_loss_fwd); the backward pass runs the fused stencil adjoint and the
transposed prolongation chain (modil_loss_bwd).  Level values live in one flat
torch tensor in the library's parameter-vector layout, so any torch optimiser
can drive the method.
"""
from __future__ import annotations

import torch

from . import modil


class ModilLoss(torch.autograd.Function):
    """loss = ModilLoss.apply(levels_flat, problem) -> 0-d float64 tensor."""

    @staticmethod
    def forward(ctx, levels, problem):
        if not levels.is_cuda or not levels.is_contiguous():
            raise ValueError("levels must be a contiguous CUDA tensor")
        dt = torch.float64 if problem.np_dtype.__name__ == "float64" else torch.float32
        if levels.dtype != dt or levels.numel() != problem.param_count():
            raise ValueError("levels must hold param_count() elements of the problem dtype")
        torch.cuda.current_stream().synchronize()  # levels are ready for the problem's stream
        terms = problem.loss_fwd(levels)
        ctx.save_for_backward(levels)
        ctx.problem = problem
        return torch.tensor(float(terms[:, 0].sum()), dtype=torch.float64, device=levels.device)

    @staticmethod
    def backward(ctx, grad_out):
        (levels,) = ctx.saved_tensors
        grads = torch.empty_like(levels)
        ctx.problem.loss_bwd(levels, float(grad_out), grads)
        ctx.problem.stream.synchronize()
        return grads, None


class ModilParameters(torch.nn.Module):
    """All levels of a problem as one flat nn.Parameter, with per-level views."""

    def __init__(self, problem, init=None):
        super().__init__()
        self.problem = problem
        dt = torch.float64 if problem.np_dtype.__name__ == "float64" else torch.float32
        n = problem.param_count()
        flat = torch.zeros(n, dtype=dt, device="cuda") if init is None else init.reshape(-1).clone()
        self.flat = torch.nn.Parameter(flat)

    def level(self, level, field=0, instance=0):
        off = self.problem.level_offset(level, field, instance)
        shape = self.problem.level_shape(level, instance)
        return self.flat[off:off + shape[0] * shape[1]].view(shape)

    def forward(self):
        return ModilLoss.apply(self.flat, self.problem)
