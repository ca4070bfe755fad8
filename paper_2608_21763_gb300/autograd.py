"""Differentiable waveforms: a torch.autograd.Function over the library.

Forward is ``s2w_waveforms``; backward is ``s2w_adjoint`` (the transpose of the
same linear map, by correlation with the conjugate spectra).  The map is
linear in the slip, so the backward pass needs only the incoming gradient:
nothing from the forward pass (seafloor spectra included) is kept for it.
"""
from __future__ import annotations

import torch


class _Waveforms(torch.autograd.Function):
    @staticmethod
    def forward(ctx, slip, context):
        ctx.context = context
        return context.waveforms(slip.contiguous())

    @staticmethod
    def backward(ctx, grad_q):
        return ctx.context.adjoint(grad_q.contiguous()), None


def waveforms(context, slip: torch.Tensor) -> torch.Tensor:
    """q = F_q D_t F_G slip for a CUDA tensor slip [B][Ns][Nt], with gradient."""
    return _Waveforms.apply(slip, context)


def misfit(context, slip: torch.Tensor, d: torch.Tensor) -> torch.Tensor:
    """0.5 ||q(slip) - d||^2 summed over the batch (differentiable)."""
    r = waveforms(context, slip) - d
    return 0.5 * (r * r).sum()
