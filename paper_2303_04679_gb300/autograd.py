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
    """loss = ModilLoss.apply(levels_flat, problem) -> 0-d float64 tensor.

    Nothing synchronises the host: the problem's stream waits for torch's
    current stream on the device, the loss is summed from the library's
    device-side loss terms, and the incoming gradient scales dL/dlevels on the
    device.  A non-finite loss shows as NaN in the returned tensor."""

    @staticmethod
    def forward(ctx, levels, problem):
        if not levels.is_cuda or not levels.is_contiguous():
            raise ValueError("levels must be a contiguous CUDA tensor")
        dt = torch.float64 if problem.np_dtype.__name__ == "float64" else torch.float32
        if levels.dtype != dt or levels.numel() != problem.param_count():
            raise ValueError("levels must hold param_count() elements of the problem dtype")
        cur = torch.cuda.current_stream()
        problem.stream.wait_stream(cur)  # levels are ready for the problem's stream
        problem.loss_fwd_async(levels)
        cur.wait_stream(problem.stream)
        if getattr(problem, "_terms_view", None) is None:
            problem._terms_view = problem.terms_device()
        ctx.save_for_backward(levels)
        ctx.problem = problem
        return problem._terms_view[:, 0].sum()

    @staticmethod
    def backward(ctx, grad_out):
        (levels,) = ctx.saved_tensors
        problem = ctx.problem
        grads = torch.empty_like(levels)
        cur = torch.cuda.current_stream()
        problem.stream.wait_stream(cur)
        problem.loss_bwd(levels, 1.0, grads)
        cur.wait_stream(problem.stream)
        return grads.mul_(grad_out.to(grads.dtype)), None


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
        n = 1
        for d in shape:  # 2-D (rows, cols) or 3-D (z, y, x)
            n *= d
        return self.flat[off:off + n].view(shape)

    def forward(self):
        return ModilLoss.apply(self.flat, self.problem)
