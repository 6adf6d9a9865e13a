"""torch.autograd wrapper of the shifted operator psi -> (Q - tau) psi (Eq. 3.6),
differentiable in the spinor fields and in the gauge links.

Forward and backward run in the library: ``qcd_apply`` (Q - tau on a batch
of fields) forwards; the spinor adjoint is the same operator (Q = Gamma5 D is
Hermitian, Sec. 2, and tau is real), and the link adjoint is
``qcd_bilinear_force``.  For a real loss L with cotangent g of the output,
dL = Re <g, (dQ) psi> along link moves U -> exp(i eps X) U (X traceless
Hermitian); the links' gradient is the tangent field i F U with F the force
of that bilinear form, summed over the batch, so that Re tr(grad^H dU)
reproduces dL for every such dU (the Riemannian gradient on SU(3); moves off
the group are not represented).

Links enter the library through ``qcd_set_gauge`` (a host copy): a forward
with ``links`` given loads them into the context, and the backward uses the
field the context holds, so run the backward before the context gets another
field.  The context must run on torch's current stream; spinors are
contiguous complex128 CUDA tensors of nrhs * V * 12 entries.
"""
import numpy as np
import torch


class ShiftedQ(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi, links, qctx, tau, lattice):
        psi = psi.contiguous()
        dims, m0, csw = lattice
        V = int(np.prod(dims))
        nrhs = psi.numel() // (12 * V)
        if nrhs * 12 * V != psi.numel():
            raise ValueError("psi must hold a whole number of fields")
        if links is not None:
            Uh = links.detach().to("cpu", torch.complex128).contiguous().numpy()
            qctx.qcd_set_gauge(Uh, dims, m0, csw)
        out = torch.empty_like(psi)
        from . import qcd
        qctx.qcd_apply(qcd.QCD_OP_Q, qcd.QCD_FP64, nrhs, psi, out, [tau] * nrhs)
        ctx.qctx, ctx.tau, ctx.V, ctx.nrhs = qctx, tau, V, nrhs
        ctx.links_shape = None if links is None else (links.shape, links.device, links.dtype)
        ctx.save_for_backward(psi)
        return out

    @staticmethod
    def backward(ctx, grad):
        from . import qcd
        (psi,) = ctx.saved_tensors
        grad = grad.contiguous()
        g_psi = g_links = None
        if ctx.needs_input_grad[0]:
            g_psi = torch.empty_like(grad)
            ctx.qctx.qcd_apply(qcd.QCD_OP_Q, qcd.QCD_FP64, ctx.nrhs, grad, g_psi, [ctx.tau] * ctx.nrhs)
        if ctx.links_shape is not None and ctx.needs_input_grad[1]:
            shape, device, dtype = ctx.links_shape
            F = torch.empty(ctx.nrhs * ctx.V * 36, dtype=torch.complex128, device=grad.device)
            ctx.qctx.qcd_bilinear_force(ctx.nrhs, grad, psi, 1, F)
            g_links = F.view(ctx.nrhs, -1).sum(dim=0).view(shape).to(device=device, dtype=dtype)
        return g_psi, g_links, None, None, None


def apply_Q(qctx, psi, tau=0.0, links=None, lattice=None):
    """(Q - tau) psi for a batch of fields, differentiable in psi and, when
    ``links`` (dims + (4, 3, 3) complex128) is given with
    ``lattice = (dims, m0, csw)``, in the links."""
    if links is not None and lattice is None:
        raise ValueError("links need lattice = (dims, m0, csw)")
    if lattice is None:
        lattice = (qctx.dims, None, None)
    return ShiftedQ.apply(psi, links, qctx, float(tau), lattice)
