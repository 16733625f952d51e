"""torch.autograd binding of the SSB phase with respect to the aberrations.

The forward is ``ssb_reconstruct`` (Eq. 3 with the aberration phase, then the
inverse transform); the backward is the hand-written adjoint ``ssb_grad``.
The spectrum G stays resident in the Reconstructor and is the only saved
state: the backward recomputes the aberration phase and re-reads G.
"""

from __future__ import annotations

import torch

from .pipeline import Reconstructor


class SSBPhase(torch.autograd.Function):
    """phi = SSBPhase.apply(theta, rec): theta float64 [5] on the GPU
    (C1, C12a, C12b, C3 in Angstrom, rot in rad), phi float32 [Ny][Nx]."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, rec: Reconstructor):
        ph, _ = rec.reconstruct(theta.detach(), phase=True)
        ctx.rec = rec
        ctx.save_for_backward(theta.detach())
        return ph[0]

    @staticmethod
    def backward(ctx, grad_phi: torch.Tensor):
        (theta,) = ctx.saved_tensors
        g = ctx.rec.grad(theta, grad_phi.contiguous())
        return g.to(theta.dtype), None


def ssb_phase(theta: torch.Tensor, rec: Reconstructor) -> torch.Tensor:
    return SSBPhase.apply(theta, rec)
