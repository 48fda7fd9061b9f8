"""Differentiable transport: torch.autograd.Function over the C ABI.

``TransportMismatch.apply(v, reg, k)`` returns ``(mismatch, m1_pred)``:
the template transported by the stationary velocity ``v`` to t = 1 (paper
Eq. 2.1b, semi-Lagrangian with RK2 characteristics) and the L2 mismatch
``1/2 ||m(1) - m1||^2``.  The backward pass is the hand-written adjoint of the
paper (Eq. 3.2 with the final condition set by the upstream gradients) plus
the time integral of the body force, computed by ``claire_mismatch_backward``;
the forward keeps the state only every ``k`` time steps and the backward
recomputes each segment (and its spatial gradient) from its checkpoint.

The gradient is the Euclidean gradient of the discrete loss, i.e. h^3 times
the L2 body force, so it is what ``torch.autograd.grad`` of the returned
scalar should be.  Like the reduced gradient of the paper it is derived
optimize-then-discretize, so it agrees with finite differences of the
discrete mismatch up to the discretization gap that shrinks under refinement.
"""
from __future__ import annotations

import torch

from . import claire


class TransportMismatch(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v: torch.Tensor, reg: "claire.Registration", checkpoint_stride: int = 2):
        v = v.detach().contiguous()
        m1_pred, mis = reg.mismatch_forward(v, checkpoint_stride)
        ctx.reg = reg
        return torch.tensor(mis, dtype=torch.float64, device=v.device), m1_pred

    @staticmethod
    def backward(ctx, grad_mis, grad_m1):
        reg = ctx.reg
        gmis = float(grad_mis) if grad_mis is not None else 0.0
        gm = None
        if grad_m1 is not None:
            gm = grad_m1.contiguous().float()
            if not torch.any(gm != 0):
                gm = None
        grad_v = reg.mismatch_backward(gmis, gm)
        return grad_v, None, None


def transport_mismatch(v, reg, checkpoint_stride: int = 2):
    """Functional form: (mismatch, m(1))."""
    return TransportMismatch.apply(v, reg, checkpoint_stride)
