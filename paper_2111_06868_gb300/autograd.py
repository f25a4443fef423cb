"""torch.autograd.Function over hq_adjoint_grad.

``energy(theta, circuit, H)`` returns E_b = <psi(theta_b)|H|psi(theta_b)> for a
(batch, P) float64 tensor of angles; its backward multiplies the incoming
gradient by dE_b/dtheta_b, which libhq computes with the adjoint reverse sweep
in the same call as the energies (so the forward already holds the gradient).
"""
from __future__ import annotations

import numpy as np
import torch

from . import hq


class AdjointEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, circuit, H, dtype, tokens, checkpoints):
        th = theta.detach().to("cpu", torch.float64).numpy()
        e, g = hq.hq_adjoint_grad(circuit, H, th, dtype=dtype, tokens=tokens, checkpoints=checkpoints)
        ctx.save_for_backward(torch.from_numpy(np.ascontiguousarray(g)))
        return torch.from_numpy(e).to(device=theta.device, dtype=theta.dtype)

    @staticmethod
    def backward(ctx, grad_e):
        (g,) = ctx.saved_tensors
        g = g.to(device=grad_e.device, dtype=grad_e.dtype)
        return grad_e[:, None] * g, None, None, None, None, None


def energy(theta: torch.Tensor, circuit, H, dtype: str = "complex64", tokens: str | None = None,
           checkpoints: int = 0) -> torch.Tensor:
    """Batched energies with an adjoint-gradient backward; theta: (batch, P) or (P,)."""
    squeeze = theta.dim() == 1
    t = theta[None, :] if squeeze else theta
    e = AdjointEnergy.apply(t, circuit, H, dtype, tokens, checkpoints)
    return e[0] if squeeze else e
