"""The autograd wrapper's gradient conventions, checked on the CPU with a
stand-in context whose calls are the oracle's dense Q - tau and the oracle's
bilinear force (host logic only: the GPU form of these checks is in
test_gpu_grad.py)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.dirac import WilsonClover, bilinear_force
from paper_2004_08146_gb300 import autograd, synth


class _OracleContext:
    """qcd_set_gauge / qcd_apply (op Q, FP64) / qcd_bilinear_force by the oracle."""

    def __init__(self, U, dims, m0, csw):
        self.qcd_set_gauge(U, dims, m0, csw)

    def qcd_set_gauge(self, U, dims, m0, csw):
        self.dims, self.m0, self.csw = tuple(dims), m0, csw
        self.op = WilsonClover(np.asarray(U).reshape(tuple(dims) + (4, 3, 3)), m0, csw)

    def qcd_apply(self, opc, prec, nrhs, inp, out, tau):
        f = inp.detach().numpy().reshape((nrhs,) + self.dims + (4, 3))
        r = np.stack([self.op.Q_shift(f[j], tau[j]) for j in range(nrhs)])
        out.copy_(torch.from_numpy(r.reshape(-1)))

    def qcd_bilinear_force(self, nvec, G, Psi, grad, F):
        g = G.detach().numpy().reshape((nvec,) + self.dims + (4, 3))
        p = Psi.detach().numpy().reshape((nvec,) + self.dims + (4, 3))
        res = []
        for j in range(nvec):
            Fj = bilinear_force(self.op, g[j], p[j])
            res.append(1j * (Fj @ self.op.U) if grad else Fj)
        F.copy_(torch.from_numpy(np.stack(res).reshape(-1)))


def _moved(U, X, eps):
    w, Y = np.linalg.eigh(X)
    E = np.einsum('...ab,...b,...cb->...ac', Y, np.exp(1j * eps * w), np.conj(Y))
    return np.einsum('...ab,...bc->...ac', E, U)


def test_backward_is_the_hermitian_operator():
    dims, tau = (2, 2, 2, 2), -0.07
    U = synth.gauge_field(dims, 0.5, 21)
    qctx = _OracleContext(U, dims, -0.3, 1.5)
    Qd = torch.from_numpy(qctx.op.dense('Q', tau))
    g = torch.from_numpy(synth.spinor(dims, 22).reshape(-1))
    p0 = synth.spinor(dims, 23).reshape(-1)
    psi = torch.from_numpy(p0.copy()).requires_grad_(True)
    torch.vdot(g, autograd.apply_Q(qctx, psi, tau)).real.backward()
    ref = torch.from_numpy(p0.copy()).requires_grad_(True)
    torch.vdot(g, Qd @ ref).real.backward()
    assert torch.max(torch.abs(psi.grad - ref.grad)).item() < 1e-12 * torch.max(torch.abs(ref.grad)).item()
    # the gradient of a real bilinear form Re <g, Q psi> is Q g
    assert torch.max(torch.abs(psi.grad - Qd @ g)).item() < 1e-12 * torch.max(torch.abs(ref.grad)).item()


def test_link_gradient_is_the_tangent_derivative():
    """L = sum_j Re <g_j, (Q - tau) psi_j> over a batch of two fields: the
    links' gradient contracted with a tangent move dU = i X U equals the
    central difference of L under U -> exp(i eps X) U (h = 1e-5)."""
    dims, tau, m0, csw = (2, 2, 2, 4), 0.11, -0.3, 1.5
    U = synth.gauge_field(dims, 0.5, 31)
    qctx = _OracleContext(U, dims, m0, csw)
    g = torch.from_numpy(synth.spinor(dims, 32, nvec=2).reshape(-1))
    psi = torch.from_numpy(synth.spinor(dims, 33, nvec=2).reshape(-1)).requires_grad_(True)
    links = torch.from_numpy(U.copy()).requires_grad_(True)
    L = torch.vdot(g, autograd.apply_Q(qctx, psi, tau, links=links, lattice=(dims, m0, csw))).real
    L.backward()
    G = links.grad.numpy()
    gs = g.numpy().reshape((2,) + dims + (4, 3))
    ps = psi.detach().numpy().reshape((2,) + dims + (4, 3))
    h = 1e-5
    for X in synth.su3_directions(dims, 34, 3):
        dU = 1j * np.einsum('...ab,...bc->...ac', X, U)
        got = np.real(np.vdot(G, dU))

        def loss(eps):
            op = WilsonClover(_moved(U, X, eps), m0, csw)
            return sum(np.real(np.vdot(gs[j], op.Q_shift(ps[j], tau))) for j in range(2))
        fd = (loss(h) - loss(-h)) / (2 * h)
        assert abs(got - fd) <= 1e-7 * max(abs(fd), 1.0), (got, fd)
