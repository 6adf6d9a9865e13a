"""GPU eigenvalue derivatives along su(3) link directions (the differentiation
form of the operator of Eq. 2.5 plus the clover term) against the oracle's
product-rule tangent (1e-12 relative) and against central differences of
dense eigenvalues (1e-6 relative), through the C ABI."""
import numpy as np
import pytest

from oracle.dirac import WilsonClover, eigenvalue_derivative
from paper_2004_08146_gb300 import synth
from gpu_util import make_ctx, dev, host, torch_cuda

pytestmark = pytest.mark.gpu


def _moved_links(U, X, eps):
    w, Y = np.linalg.eigh(X)
    E = np.einsum('...ab,...b,...cb->...ac', Y, np.exp(1j * eps * w), np.conj(Y))
    return np.einsum('...ab,...bc->...ac', E, U)


@pytest.mark.parametrize("dims,antip", [((4, 4, 2, 2), True), ((2, 4, 4, 2), False), ((4, 4, 4, 4), True)])
def test_derivative_matches_oracle(dims, antip):
    """v^H Gamma5 (dD/deps) v / v^H v on random spinors (any v: the quantity is
    defined for all), every direction and boundary phase exercised."""
    torch_cuda()
    U = synth.gauge_field(dims, 0.5, 101)
    X = synth.su3_directions(dims, 102, 1)[0]
    op = WilsonClover(U, -0.3, 1.5, antiperiodic_t=antip)
    ctx = make_ctx(U, dims, -0.3, 1.5, antiperiodic_t=int(antip))
    psi = synth.spinor(dims, 103, nvec=5)
    got = ctx.qcd_eig_derivative(X, 5, dev(psi))
    ref = np.array([eigenvalue_derivative(op, X, psi[j]) for j in range(5)])
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_hellmann_feynman_against_eigenvalue_differences():
    """The 4^4 workload field: derivatives of the six smallest |lambda| along two
    random directions against central differences (h = 1e-5) of the dense
    eigenvalues at U(+h) and U(-h)."""
    torch_cuda()
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 1001)
    op = WilsonClover(U, -0.2, 1.0)
    w, Y = np.linalg.eigh(op.dense('Q'))
    ks = np.argsort(np.abs(w))[:6]
    ctx = make_ctx(U, dims, -0.2, 1.0)
    vecs = np.ascontiguousarray(Y[:, ks].T)
    h = 1e-5
    for X in synth.su3_directions(dims, 111, 2):
        got = ctx.qcd_eig_derivative(X, len(ks), dev(vecs))
        wp = np.linalg.eigvalsh(WilsonClover(_moved_links(U, X, h), -0.2, 1.0).dense('Q'))
        wm = np.linalg.eigvalsh(WilsonClover(_moved_links(U, X, -h), -0.2, 1.0).dense('Q'))
        for j, k in enumerate(ks):
            assert np.min(np.abs(np.delete(w, k) - w[k])) > 1e-6
            fd = (wp[k] - wm[k]) / (2 * h)
            assert abs(got[j] - fd) <= 1e-6 * max(abs(fd), 1e-3), (k, got[j], fd)


@pytest.mark.parametrize("dims,antip,csw", [((4, 4, 2, 2), True, 1.5), ((2, 4, 4, 2), False, 1.5),
                                            ((4, 2, 2, 4), True, 0.0)])
def test_force_matches_oracle(dims, antip, csw):
    """Per-link force of v^H Q v / v^H v, element by element against the
    oracle (1e-12 of the largest entry), every direction, both boundary
    phases and the Wilson case c_sw = 0."""
    torch = torch_cuda()
    from oracle.dirac import eigenvalue_force
    U = synth.gauge_field(dims, 0.5, 131)
    op = WilsonClover(U, -0.3, csw, antiperiodic_t=antip)
    ctx = make_ctx(U, dims, -0.3, csw, antiperiodic_t=int(antip))
    psi = synth.spinor(dims, 132, nvec=3)
    nl = 36 * int(np.prod(dims))
    F = torch.zeros(3 * nl, dtype=torch.complex128, device="cuda")
    ctx.qcd_eig_force(3, dev(psi), F)
    got = host(F).reshape((3,) + dims + (4, 3, 3))
    for j in range(3):
        ref = eigenvalue_force(op, psi[j])
        assert np.max(np.abs(got[j] - ref)) < 1e-12 * np.max(np.abs(ref)), j


def test_force_contracts_to_derivative():
    """On the 4^4 field: sum tr(X F) of the GPU force equals the GPU
    directional derivative along each of three directions (1e-12)."""
    torch = torch_cuda()
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 141)
    ctx = make_ctx(U, dims, -0.2, 1.0)
    psi = synth.spinor(dims, 142, nvec=4)
    nl = 36 * int(np.prod(dims))
    F = torch.zeros(4 * nl, dtype=torch.complex128, device="cuda")
    V = dev(psi)
    ctx.qcd_eig_force(4, V, F)
    Fh = host(F).reshape(4, -1, 3, 3)
    assert np.max(np.abs(Fh - np.conj(np.swapaxes(Fh, -1, -2)))) < 1e-14 * np.max(np.abs(Fh))
    assert np.max(np.abs(np.trace(Fh, axis1=-2, axis2=-1))) < 1e-14 * np.max(np.abs(Fh))
    for X in synth.su3_directions(dims, 143, 3):
        der = ctx.qcd_eig_derivative(X, 4, V)
        con = np.einsum('kiab,iba->k', Fh, X.reshape(-1, 3, 3)).real
        assert np.max(np.abs(con - der)) < 1e-12 * np.max(np.abs(der))


def test_autograd_adjoint_is_the_operator():
    """psi.grad of Re <g, (Q - tau) psi> through the autograd wrapper equals
    torch's own autograd through the oracle's dense Q - tau."""
    torch = torch_cuda()
    from paper_2004_08146_gb300 import autograd
    dims, tau = (2, 4, 2, 2), 0.13
    U = synth.gauge_field(dims, 0.5, 151)
    op = WilsonClover(U, -0.3, 1.5)
    ctx = make_ctx(U, dims, -0.3, 1.5)
    p0 = synth.spinor(dims, 152).reshape(-1)
    g = synth.spinor(dims, 153).reshape(-1)
    psi = dev(p0).requires_grad_(True)
    torch.vdot(dev(g), autograd.apply_Q(ctx, psi, tau)).real.backward()
    pr = torch.from_numpy(p0.copy()).requires_grad_(True)
    torch.vdot(torch.from_numpy(g), torch.from_numpy(op.dense('Q', tau)) @ pr).real.backward()
    assert np.max(np.abs(host(psi.grad) - pr.grad.numpy())) < 1e-12 * np.max(np.abs(pr.grad.numpy()))


@pytest.mark.parametrize("dims,antip,csw", [((4, 4, 2, 2), True, 1.5), ((2, 4, 4, 2), False, 1.5),
                                            ((4, 2, 2, 4), True, 0.0)])
def test_bilinear_force_matches_oracle(dims, antip, csw):
    """Force of Re <g, Q psi> for distinct g, psi (the link adjoint of the
    autograd wrapper), element by element against the oracle (1e-12 of the
    largest entry); the gradient form equals i F U."""
    torch = torch_cuda()
    from oracle.dirac import bilinear_force
    U = synth.gauge_field(dims, 0.5, 171)
    op = WilsonClover(U, -0.3, csw, antiperiodic_t=antip)
    ctx = make_ctx(U, dims, -0.3, csw, antiperiodic_t=int(antip))
    g = synth.spinor(dims, 172, nvec=3)
    psi = synth.spinor(dims, 173, nvec=3)
    nl = 36 * int(np.prod(dims))
    F = torch.zeros(3 * nl, dtype=torch.complex128, device="cuda")
    Gr = torch.zeros_like(F)
    ctx.qcd_bilinear_force(3, dev(g), dev(psi), 0, F)
    ctx.qcd_bilinear_force(3, dev(g), dev(psi), 1, Gr)
    got = host(F).reshape((3,) + dims + (4, 3, 3))
    gr = host(Gr).reshape((3,) + dims + (4, 3, 3))
    for j in range(3):
        ref = bilinear_force(op, g[j], psi[j])
        assert np.max(np.abs(got[j] - ref)) < 1e-12 * np.max(np.abs(ref)), j
        assert np.max(np.abs(gr[j] - 1j * (ref @ U))) < 1e-12 * np.max(np.abs(ref)), j


def test_autograd_links_central_differences_16c4():
    """The differentiation workload: 16^4 field (eps 0.5, c_sw 1.5), 8 random
    complex128 spinors psi_j and cotangents g_j, L = sum_j Re <g_j, (Q - tau)
    psi_j> through the autograd wrapper with the links as an input.  The links'
    gradient contracted with dU = i X U matches the central difference
    (h = 1e-5) of L under U -> exp(i eps X) U along 16 random su(3) directions
    to 1e-6 relative; the spinor gradient is (Q - tau) g."""
    torch = torch_cuda()
    from paper_2004_08146_gb300 import autograd
    from paper_2004_08146_gb300 import workloads
    w = workloads.get("c5_16c4")
    dims, tau, m0, csw = tuple(w["dims"]), 0.05, w["m0"], w["csw"]
    U = synth.gauge_field(dims, w["eps"], w["seed"])
    ctx = make_ctx(U, dims, m0, csw)
    nrhs = 8
    g = dev(synth.spinor(dims, 181, nvec=nrhs))
    psi = dev(synth.spinor(dims, 182, nvec=nrhs)).requires_grad_(True)
    links = torch.from_numpy(U.copy()).requires_grad_(True)
    L = torch.vdot(g, autograd.apply_Q(ctx, psi, tau, links=links, lattice=(dims, m0, csw))).real
    L.backward()
    Gl = links.grad.numpy()
    # spinor gradient
    Qg = torch.empty_like(g)
    ctx.qcd_apply(1, 0, nrhs, g, Qg, [tau] * nrhs)
    assert (psi.grad - Qg).abs().max().item() < 1e-12 * Qg.abs().max().item()
    out = torch.empty_like(g)
    h = 1e-5

    def loss(Um):
        ctx.qcd_set_gauge(Um, dims, m0, csw)
        ctx.qcd_apply(1, 0, nrhs, psi.detach(), out, [tau] * nrhs)
        torch.cuda.synchronize()
        return torch.vdot(g, out).real.item()

    def moved(X, eps):   # exp(i eps X) U to O(eps^4) ~ 1e-20
        X2 = np.einsum('...ab,...bc->...ac', X, X)
        X3 = np.einsum('...ab,...bc->...ac', X2, X)
        E = np.eye(3) + 1j * eps * X - 0.5 * eps * eps * X2 - 1j * eps ** 3 / 6 * X3
        return np.einsum('...ab,...bc->...ac', E, U)

    for d in range(16):
        X = synth.su3_directions(dims, 2000 + d, 1)[0]
        dU = 1j * np.einsum('...ab,...bc->...ac', X, U)
        got = np.real(np.vdot(Gl, dU))
        fd = (loss(moved(X, h)) - loss(moved(X, -h))) / (2 * h)
        assert abs(got - fd) <= 1e-6 * abs(fd), (d, got, fd)
    ctx.close()
