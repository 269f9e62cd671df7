"""Differentiable persistence diagrams as a torch.autograd.Function.

Forward: the VR filtrations of the clouds are built from grid-rounded coordinates, reduced with
Algorithm 2 and turned into per-cloud losses sum (d - b)^2 over the finite pairs of one
dimension, b and d being the fp32 lengths of the realising edges (all in the library's
kernels). Backward: the library's scatter kernel adds each pair's gradient to the four
realising points. The pairing itself is exact and piecewise constant, so it gets no gradient.
"""
from __future__ import annotations

import torch

from .native import Context


class DiagramLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coords, cloud_offsets, dim, context):
        context.build_filtration_f32(coords.detach(), cloud_offsets, max_dim=dim + 1)
        st = context.reduce()
        if not st["converged"]:
            raise RuntimeError("reduction did not converge")
        loss = context.diagram_loss(coords.detach(), dim)
        ctx.save_for_backward(coords)
        ctx.dim = dim
        ctx.context = context
        ctx.build = context.builds  # the filtration this loss was computed on
        return loss[:-1].clone()

    @staticmethod
    def backward(ctx, grad_loss):
        (coords,) = ctx.saved_tensors
        if ctx.context.builds != ctx.build:
            # the gradient scatters through the context's current pairing: after another
            # build it would belong to a different filtration
            raise RuntimeError("the context was rebuilt between this loss's forward and backward;"
                               " give each loss its own Context")
        grad = ctx.context.diagram_backward(coords.detach(), grad_loss, ctx.dim)
        return grad, None, None, None


def diagram_loss(coords: torch.Tensor, cloud_offsets=None, dim: int = 1,
                 context: Context | None = None) -> torch.Tensor:
    """Per-cloud diagram losses (differentiable with respect to ``coords``)."""
    if context is None:
        context = Context()
    return DiagramLoss.apply(coords, cloud_offsets, dim, context)
