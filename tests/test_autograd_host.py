"""The autograd wrapper's gradient convention, checked on the CPU with a
stand-in context whose qcd_apply_Q multiplies by the oracle's dense Q - tau
(host logic only: the GPU form of this check is in test_gpu_grad.py)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.dirac import WilsonClover
from paper_2004_08146_gb300 import autograd, synth


class _DenseContext:
    def __init__(self, op, tau):
        self.Q = torch.from_numpy(op.dense('Q', tau))
        self.tau = tau

    def qcd_apply_Q(self, inp, out, tau):
        assert tau == self.tau
        out.copy_(self.Q @ inp)


def test_backward_is_the_hermitian_operator():
    dims, tau = (2, 2, 2, 2), -0.07
    op = WilsonClover(synth.gauge_field(dims, 0.5, 21), -0.3, 1.5)
    qctx = _DenseContext(op, tau)
    g = torch.from_numpy(synth.spinor(dims, 22).reshape(-1))
    p0 = synth.spinor(dims, 23).reshape(-1)
    psi = torch.from_numpy(p0.copy()).requires_grad_(True)
    torch.vdot(g, autograd.apply_Q(qctx, psi, tau)).real.backward()
    ref = torch.from_numpy(p0.copy()).requires_grad_(True)
    torch.vdot(g, qctx.Q @ ref).real.backward()
    assert torch.max(torch.abs(psi.grad - ref.grad)).item() < 1e-12 * torch.max(torch.abs(ref.grad)).item()
    # the gradient of a real bilinear form Re <g, Q psi> is Q g
    assert torch.max(torch.abs(psi.grad - qctx.Q @ g)).item() < 1e-12 * torch.max(torch.abs(ref.grad)).item()
