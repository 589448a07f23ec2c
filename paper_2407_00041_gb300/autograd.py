"""torch.autograd.Function around D psi.

Forward: eta = D psi (dd_apply).  Backward, for a real loss L and the incoming
gradient phi = dL/dRe eta + i dL/dIm eta:
  grad psi = D^H phi          (dd_apply with DD_OP_DH; D^H = gamma5 D gamma5)
  grad U   = G = dL/dRe U + i dL/dIm U of Re <phi, D psi>   (dd_force)
The link derivative recomputes the projected half-spinors of phi and psi;
nothing from the forward pass is stored except psi itself.

``U`` must be the links the operator handle was built from; it is an input
only so that autograd can route its gradient.
"""
from __future__ import annotations

import torch

from . import binding as B


class DiracApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi, U, op, prec, with_clover):
        psi = psi.contiguous()
        nrhs = psi.shape[0]
        out = torch.empty_like(psi)
        op.apply(B.DD_OP_D, prec, psi, out, nrhs)
        ctx.save_for_backward(psi)
        ctx.op, ctx.prec, ctx.with_clover, ctx.nrhs, ctx.ushape = op, prec, with_clover, nrhs, U.shape
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (psi,) = ctx.saved_tensors
        phi = grad_out.contiguous()
        grad_psi = grad_U = None
        if ctx.needs_input_grad[0]:
            grad_psi = torch.empty_like(phi)
            ctx.op.apply(B.DD_OP_DH, ctx.prec, phi, grad_psi, ctx.nrhs)
        if ctx.needs_input_grad[1]:
            grad_U = torch.empty(ctx.ushape, dtype=torch.complex128, device=phi.device)
            fprec = B.DD_PREC_F64 if ctx.prec == B.DD_PREC_F64 else B.DD_PREC_F32
            ctx.op.force(fprec, phi, psi, ctx.nrhs, ctx.with_clover, G=grad_U)
        return grad_psi, grad_U, None, None, None


def dirac(psi, U, op, prec=B.DD_PREC_F64, with_clover=True):
    """eta = D psi with autograd support for psi ([nrhs, V, 4, 3] complex128 on
    the device) and U ([V, 4, 3, 3] complex128).  with_clover=False holds the
    self coupling fixed in the link derivative."""
    return DiracApply.apply(psi, U, op, prec, with_clover)


def su3_force(op, phi, psi, with_clover=True, prec=B.DD_PREC_F64):
    """(G, F): link derivative of Re <phi, D psi> and its su(3) projection
    F = P(G U^H), both complex128 [V, 4, 3, 3] on the device."""
    V = op.lattice.V
    G = torch.empty((V, 4, 3, 3), dtype=torch.complex128, device=phi.device)
    F = torch.empty_like(G)
    op.force(prec, phi.contiguous(), psi.contiguous(), phi.shape[0], with_clover, G=G, F=F)
    return G, F
