"""GPU eigenvalue derivatives along su(3) link directions (the differentiation
form of the operator of Eq. 2.5 plus the clover term) against the oracle's
product-rule tangent (1e-12 relative) and against central differences of
dense eigenvalues (1e-6 relative), through the C ABI."""
import numpy as np
import pytest

from oracle.dirac import WilsonClover, eigenvalue_derivative
from paper_2004_08146_gb300 import synth
from gpu_util import make_ctx, dev, torch_cuda

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
