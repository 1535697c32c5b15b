"""KL(P || Q^H) as a torch.autograd.Function.

forward  = hts_kl   (Eq. KLDivergence with the hyperbolic q of Eq.
           LowDimensionalProbabilityHyperbolic; exact Z at theta = 0, tree Z
           otherwise),
backward = hts_grad (the gradient kernels: Eq. KLGradientHyperbolic in the
           split form of Eq. KlGradientHyperbolicSplit, exaggeration 1),
scaled by the incoming gradient.  At theta = 0 the backward is the exact
derivative of the forward; at theta > 0 it is the Barnes-Hut approximation
of it.  Both run in the CUDA library; this module only moves tensors.

The model's P is used as set; each call copies y into the model with
hts_set_Y (which also resets the model's velocity, so do not interleave these
calls with a running hts_step optimisation on the same model).  The CO-SNE
term, if switched on in the model, would enter the backward but not the
forward; switch it off for this use.
"""
from __future__ import annotations

import torch

from .api import HyperbolicTSNE


class KLFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y: torch.Tensor, model: HyperbolicTSNE, theta: float = 0.0):
        if y.dtype != torch.float64 or y.dim() != 2 or y.shape[1] != 2:
            raise TypeError("y must be an (n, 2) float64 tensor")
        yc = y.detach().contiguous()
        model.set_Y(yc)
        value = model.kl(theta)
        ctx.model = model
        ctx.theta = float(theta)
        ctx.save_for_backward(yc)
        return torch.tensor(value, dtype=y.dtype, device=y.device)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (yc,) = ctx.saved_tensors
        model = ctx.model
        model.set_Y(yc)
        g = torch.empty_like(yc)
        if g.is_cuda:
            model.grad(ctx.theta, 1.0, out=g)
        else:
            g.copy_(torch.from_numpy(model.grad(ctx.theta, 1.0)[0]))
        return grad_out * g, None, None


def kl_divergence(y: torch.Tensor, model: HyperbolicTSNE, theta: float = 0.0) -> torch.Tensor:
    """Differentiable KL(P || Q^H) of the embedding y under `model`'s P."""
    return KLFunction.apply(y, model, theta)
