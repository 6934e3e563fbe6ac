"""The topological loss as a differentiable PyTorch function.

`topological_loss(f, field)` returns L(f), the W2^2 distance (Eq. 2, q = 2)
between the persistence diagram of `f` and the field's target diagram, every
point matched by the exact solver.  Both the forward value and the backward
gradient come from the library's kernels (`tsf_loss_and_gradient`): the
gradient is Section 4.1's per-pair contribution without the step size,
summed per vertex in fp64 and returned in the dtype of `f`.  It is the exact
derivative of L wherever a small change of `f` changes neither the pairing
nor the matching (L is piecewise quadratic in f).
"""
from __future__ import annotations

import torch

from . import Field


class _TopologicalLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, field):
        if f.dim() != 3 or tuple(f.shape) != field.shape:
            raise ValueError("f must have the field's (Lz, Ly, Lx) shape")
        values = f.detach().to(torch.float32).contiguous()
        grad = torch.empty(values.shape, dtype=torch.float64, device=values.device)
        loss, _ = field.loss_and_grad(values, grad)
        ctx.save_for_backward(grad)
        ctx.dtype = f.dtype
        return torch.tensor(loss, dtype=torch.float64, device=f.device)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return (g * grad).to(ctx.dtype), None


def topological_loss(f: torch.Tensor, field: Field) -> torch.Tensor:
    """L(f) as a float64 scalar tensor with a backward pass (see module doc)."""
    return _TopologicalLoss.apply(f, field)
