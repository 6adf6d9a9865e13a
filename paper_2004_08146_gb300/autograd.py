"""torch.autograd wrapper of the shifted operator Q - tau (Eq. 3.6).

Forward and backward both run the library's Wilson-clover stencil through
``qcd_apply_Q``.  Q = Gamma5 D is Hermitian (Sec. 2) and tau is real, so the
adjoint of psi -> (Q - tau) psi with respect to the spinor is the same
operator: the backward pass applies it to the incoming gradient.  The link
derivative of an eigenvalue is the per-link force ``qcd_eig_force`` (a field,
not an autograd input: links enter the library through ``qcd_set_gauge``).

The context must run on the stream torch uses for these tensors (create it
with ``stream=torch.cuda.current_stream().cuda_stream``); spinors are
contiguous complex128 CUDA tensors of V*12 entries.
"""
import torch


class ShiftedQ(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi, qctx, tau):
        psi = psi.contiguous()
        out = torch.empty_like(psi)
        qctx.qcd_apply_Q(psi, out, tau)
        ctx.qctx = qctx
        ctx.tau = tau
        return out

    @staticmethod
    def backward(ctx, grad):
        grad = grad.contiguous()
        out = torch.empty_like(grad)
        ctx.qctx.qcd_apply_Q(grad, out, ctx.tau)
        return out, None, None


def apply_Q(qctx, psi, tau=0.0):
    """(Q - tau) psi, differentiable in psi."""
    return ShiftedQ.apply(psi, qctx, float(tau))
