"""Pins of the oracle's Wilson-clover operator against what the paper and the
mathematics fix (no GPU).  Each test names the passage or the closed form it
checks."""
import itertools

import numpy as np
import pytest

from oracle.dirac import GAMMA, GAMMA5, WilsonClover, clover_field, sigma_munu
from paper_2004_08146_gb300 import synth


def _field(op, v):
    return op.shape_field(v)


# ------------------------------------------------------------ gamma matrices
def test_gamma_clifford_and_gamma5():
    """Eq. 2.3 (Clifford relations), Hermiticity, Eq. 2.4 (gamma5 anticommutes
    with every gamma_mu) and the representation gamma5 = diag(I2, -I2) that
    Sec. 2 fixes."""
    for mu in range(4):
        assert np.allclose(GAMMA[mu], GAMMA[mu].conj().T, atol=0)
        for nu in range(4):
            anti = GAMMA[mu] @ GAMMA[nu] + GAMMA[nu] @ GAMMA[mu]
            assert np.allclose(anti, 2.0 * (mu == nu) * np.eye(4), atol=1e-15)
        assert np.allclose(GAMMA5 @ GAMMA[mu], -GAMMA[mu] @ GAMMA5, atol=1e-15)
    assert np.allclose(GAMMA5, np.diag([1, 1, -1, -1]), atol=1e-15)


# ------------------------------------------------------------ free field
def _free_spectrum(dims, m0, antiperiodic_t):
    """Closed form for U = 1: plane waves with momenta p_mu diagonalise Eq. 2.5,
    D(p) = m0 + sum_mu (1 - cos p_mu) + i sum_mu gamma_mu sin p_mu, hence
    Q(p)^2 = (M(p)^2 + sum sin^2 p_mu) I and Q has the eigenvalues
    +-sqrt(M^2 + s^2), each 6-fold (2 spins x 3 colours)."""
    lam = []
    ranges = [range(L) for L in dims]
    for n in itertools.product(*ranges):
        p = []
        for mu, (nmu, L) in enumerate(zip(n, dims)):
            if mu == 0 and antiperiodic_t:
                p.append((2 * nmu + 1) * np.pi / L)
            else:
                p.append(2 * np.pi * nmu / L)
        M = m0 + sum(1 - np.cos(q) for q in p)
        s2 = sum(np.sin(q) ** 2 for q in p)
        e = np.sqrt(M * M + s2)
        lam += [e] * 6 + [-e] * 6
    return np.sort(lam)


@pytest.mark.parametrize("dims,antip", [((4, 2, 2, 2), True), ((2, 4, 2, 2), False),
                                        ((6, 2, 2, 4), True)])
def test_free_field_spectrum_small(dims, antip):
    op = WilsonClover(synth.unit_gauge(dims), -0.2, 1.0, antiperiodic_t=antip)
    ev = np.linalg.eigvalsh(op.dense('Q'))
    assert np.max(np.abs(np.sort(ev) - _free_spectrum(dims, -0.2, antip))) < 1e-12


@pytest.mark.slow
def test_free_field_spectrum_4x4x4x4():
    """4^4, m0 = -0.2, antiperiodic time: smallest |lambda| = 0.71318241
    (24-fold) and the spectrum spans [-7.5403, 7.5403] by the closed form."""
    dims = (4, 4, 4, 4)
    op = WilsonClover(synth.unit_gauge(dims), -0.2, 1.0)
    ev = np.sort(np.linalg.eigvalsh(op.dense('Q')))
    ref = _free_spectrum(dims, -0.2, True)
    assert np.max(np.abs(ev - ref)) < 1e-12
    assert abs(np.min(np.abs(ev)) - 0.71318241) < 1e-8
    assert np.sum(np.abs(np.abs(ev) - np.min(np.abs(ev))) < 1e-10) == 24


def test_free_field_clover_vanishes():
    """U = 1: every plaquette is the identity, F = 0, the clover term is 0."""
    C = clover_field(synth.unit_gauge((2, 2, 2, 2)), 1.7)
    assert np.max(np.abs(C)) == 0.0


# ------------------------------------------------------------ symmetries
@pytest.fixture(scope="module")
def rough_op():
    dims = (4, 2, 4, 2)
    U = synth.gauge_field(dims, 0.5, 4242)
    return WilsonClover(U, -0.3, 1.5)


def test_links_are_su3(rough_op):
    U = rough_op.U
    eye = np.eye(3)
    assert np.max(np.abs(U @ np.conj(np.swapaxes(U, -1, -2)) - eye)) < 1e-13
    assert np.max(np.abs(np.linalg.det(U) - 1.0)) < 1e-13


def test_Q_hermitian_apply(rough_op):
    """<x, Q y> = <Q x, y> (Eq. 2.7, Q = Gamma5 D Hermitian) to 1e-14 relative."""
    op = rough_op
    x = synth.spinor(op.dims, 1)
    y = synth.spinor(op.dims, 2)
    a = np.vdot(x, op.Q(y))
    b = np.vdot(op.Q(x), y)
    assert abs(a - b) <= 1e-14 * max(abs(a), np.linalg.norm(x) * np.linalg.norm(op.Q(y)))


def test_gamma5_symmetry_dense():
    """Gamma5 D = (Gamma5 D)^H, i.e. D^H = Gamma5 D Gamma5 (Eq. 2.7), dense."""
    dims = (2, 2, 2, 4)
    op = WilsonClover(synth.gauge_field(dims, 0.6, 7), 0.1, 1.2)
    D = op.dense('D')
    G5 = np.kron(np.eye(int(np.prod(dims))), np.kron(GAMMA5, np.eye(3)))
    assert np.max(np.abs(D.conj().T - G5 @ D @ G5)) < 1e-13
    Q = op.dense('Q')
    assert np.max(np.abs(Q - Q.conj().T)) < 1e-13
    assert np.max(np.abs(Q - G5 @ D)) < 1e-14


def test_hop_entries_match_eq_2_6():
    """Matrix entries of Eq. 2.6: (D)_{x,x+mu} = -1/2 (I - gamma_mu) (x) U_mu(x)
    and (D)_{x+mu,x} = -1/2 (I + gamma_mu) (x) U_mu(x)^H, read off the dense
    matrix at an interior pair of sites (no boundary phase)."""
    dims = (4, 4, 2, 2)
    U = synth.gauge_field(dims, 0.7, 99)
    op = WilsonClover(U, 0.0, 0.0, antiperiodic_t=False)
    D = op.dense('D')
    x = (1, 2, 0, 1)
    for mu in range(4):
        y = list(x)
        y[mu] = (y[mu] + 1) % dims[mu]
        ix = np.ravel_multi_index(x, dims)
        iy = np.ravel_multi_index(tuple(y), dims)
        Umu = U[x + (mu,)]
        blk_fwd = D[12 * ix:12 * ix + 12, 12 * iy:12 * iy + 12]
        blk_bwd = D[12 * iy:12 * iy + 12, 12 * ix:12 * ix + 12]
        if dims[mu] == 2:   # x+mu and x-mu coincide: both hops land in one block
            Umu_b = U[tuple(y) + (mu,)]
            ref_f = -0.5 * np.kron(np.eye(4) - GAMMA[mu], Umu) - 0.5 * np.kron(np.eye(4) + GAMMA[mu], Umu_b.conj().T)
            assert np.max(np.abs(blk_fwd - ref_f)) < 1e-14
            continue
        assert np.max(np.abs(blk_fwd + 0.5 * np.kron(np.eye(4) - GAMMA[mu], Umu))) < 1e-14
        assert np.max(np.abs(blk_bwd + 0.5 * np.kron(np.eye(4) + GAMMA[mu], Umu.conj().T))) < 1e-14


def test_antiperiodic_phase_dense():
    """Antiperiodic time: the hop entries across t = L0-1 -> 0 carry -1."""
    dims = (4, 2, 2, 2)
    U = synth.gauge_field(dims, 0.4, 5)
    Dp = WilsonClover(U, 0.0, 0.0, antiperiodic_t=False).dense('D')
    Da = WilsonClover(U, 0.0, 0.0, antiperiodic_t=True).dense('D')
    diff = Da - Dp
    V = int(np.prod(dims))
    t = np.unravel_index(np.arange(V), dims)[0]
    for i in range(V):
        for j in range(V):
            blk = diff[12 * i:12 * i + 12, 12 * j:12 * j + 12]
            crosses = (t[i] == dims[0] - 1 and t[j] == 0) or (t[i] == 0 and t[j] == dims[0] - 1)
            if crosses:
                Pblk = Dp[12 * i:12 * i + 12, 12 * j:12 * j + 12]
                assert np.max(np.abs(blk + 2 * Pblk)) < 1e-14
            else:
                assert np.max(np.abs(blk)) == 0.0


def test_gauge_covariance(rough_op):
    """U_mu(x) -> Om(x) U_mu(x) Om(x+mu)^H gives D -> G D G^H with
    G = diag(I4 (x) Om(x)): apply-level agreement to 1e-13 relative, hence an
    invariant spectrum."""
    op = rough_op
    dims = op.dims
    Om = synth.random_su3(dims, 31)
    Ut = np.empty_like(op.U)
    for mu in range(4):
        Om_fwd = np.roll(Om, -1, axis=mu)
        Ut[..., mu, :, :] = Om @ op.U[..., mu, :, :] @ np.conj(np.swapaxes(Om_fwd, -1, -2))
    opt = WilsonClover(Ut, op.m0, op.csw)
    psi = synth.spinor(dims, 3)
    G = lambda f: np.einsum('...ab,...sb->...sa', Om, f)
    lhs = opt.Q(G(psi))
    rhs = G(op.Q(psi))
    assert np.linalg.norm(lhs - rhs) <= 1e-13 * np.linalg.norm(rhs)


@pytest.mark.slow
def test_gauge_covariance_spectrum():
    dims = (2, 2, 2, 4)
    op = WilsonClover(synth.gauge_field(dims, 0.5, 8), -0.1, 1.3)
    Om = synth.random_su3(dims, 9)
    Ut = np.empty_like(op.U)
    for mu in range(4):
        Ut[..., mu, :, :] = Om @ op.U[..., mu, :, :] @ np.conj(np.swapaxes(np.roll(Om, -1, axis=mu), -1, -2))
    e1 = np.linalg.eigvalsh(op.dense('Q'))
    e2 = np.linalg.eigvalsh(WilsonClover(Ut, -0.1, 1.3).dense('Q'))
    assert np.max(np.abs(e1 - e2)) < 1e-12


# ------------------------------------------------------------ clover
def test_clover_hermitian_chiral_blocks(rough_op):
    """The clover term is Hermitian and commutes with gamma5: it consists of
    two 6x6 blocks per site (Sec. 4, Table 1 discussion)."""
    C = rough_op.C
    assert np.max(np.abs(C - np.conj(np.swapaxes(C, -1, -2)))) < 1e-14
    assert np.max(np.abs(C[..., :6, 6:])) == 0.0
    assert np.max(np.abs(C[..., 6:, :6])) == 0.0


def test_clover_constant_abelian_field():
    """Hand-computable field strength: U_1(x) = exp(i B x_2 T) with
    T = diag(1, -1, 0), B = 2 pi n / L_2 and all other links 1.  Every (1,2)
    plaquette leaf equals exp(-i B T), so F_12 = -i sin(B T), the other planes
    vanish, and the clover matrix is (c_sw/2) sigma_12 (x) diag(sin B, -sin B, 0)."""
    dims = (2, 2, 4, 2)
    B = 2 * np.pi * 1 / dims[2]
    U = synth.unit_gauge(dims)
    x2 = np.indices(dims)[2]
    ph = np.exp(1j * B * x2)
    U[..., 1, 0, 0] = ph
    U[..., 1, 1, 1] = np.conj(ph)
    csw = 1.3
    C = clover_field(U, csw)
    ref = 0.5 * csw * np.kron(sigma_munu(1, 2), np.diag([np.sin(B), -np.sin(B), 0.0]))
    assert np.max(np.abs(C - ref)) < 1e-14


def _moved_links(U, X, eps):
    """U_mu(x) -> exp(i eps X_mu(x)) U_mu(x), the exponential through numpy's
    Hermitian eigendecomposition."""
    w, Y = np.linalg.eigh(X)
    E = np.einsum('...ab,...b,...cb->...ac', Y, np.exp(1j * eps * w), np.conj(Y))
    return np.einsum('...ab,...bc->...ac', E, U)


def test_operator_tangent_matches_central_difference():
    """dD/deps along a random su(3) direction field (product rule through the
    hop terms and every clover leaf) against a central difference of the whole
    operator rebuilt at U(+h) and U(-h), antiperiodic time, csw = 1.5."""
    from oracle.dirac import operator_tangent
    dims = (4, 4, 2, 2)
    U = synth.gauge_field(dims, 0.5, 81)
    X = synth.su3_directions(dims, 82, 1)[0]
    psi = synth.spinor(dims, 83)
    op = WilsonClover(U, -0.3, 1.5)
    got = operator_tangent(op, X)(psi)
    h = 1e-4
    Dp = WilsonClover(_moved_links(U, X, h), -0.3, 1.5).D(psi)
    Dm = WilsonClover(_moved_links(U, X, -h), -0.3, 1.5).D(psi)
    fd = (Dp - Dm) / (2 * h)
    assert np.linalg.norm(got - fd) < 1e-7 * np.linalg.norm(fd)


def test_hellmann_feynman_matches_eigenvalue_difference():
    """d lambda_k / d eps (Hellmann-Feynman with the operator tangent) against a
    central difference of the dense eigenvalues of Q at U(+-h), for the five
    eigenvalues of smallest modulus (simple for this random field)."""
    from oracle.dirac import eigenvalue_derivative
    dims = (4, 4, 2, 2)
    U = synth.gauge_field(dims, 0.5, 91)
    X = synth.su3_directions(dims, 92, 1)[0]
    op = WilsonClover(U, -0.3, 1.5)
    w, Y = np.linalg.eigh(op.dense('Q'))
    order = np.argsort(np.abs(w))[:5]
    h = 1e-5
    wp = np.linalg.eigvalsh(WilsonClover(_moved_links(U, X, h), -0.3, 1.5).dense('Q'))
    wm = np.linalg.eigvalsh(WilsonClover(_moved_links(U, X, -h), -0.3, 1.5).dense('Q'))
    for k in order:
        assert np.min(np.abs(np.delete(w, k) - w[k])) > 1e-6          # simple eigenvalue
        fd = (wp[k] - wm[k]) / (2 * h)                                  # eigvalsh keeps the ascending order
        hf = eigenvalue_derivative(op, X, Y[:, k])
        assert abs(hf - fd) <= 1e-6 * max(abs(fd), 1e-3)


@pytest.mark.parametrize("dims,antip,csw", [((2, 2, 2, 2), True, 1.5), ((4, 2, 2, 4), True, 1.5),
                                            ((2, 4, 2, 2), False, 0.0), ((4, 4, 2, 2), False, 1.2)])
def test_force_contracts_to_directional_derivative(dims, antip, csw):
    """sum_{x,mu} tr(X_mu(x) F_mu(x)) of the per-link force equals the
    product-rule directional derivative (itself pinned by central differences
    above) for random su(3) directions; F is traceless Hermitian."""
    from oracle.dirac import eigenvalue_derivative, eigenvalue_force
    U = synth.gauge_field(dims, 0.5, 7)
    op = WilsonClover(U, -0.3, csw, antiperiodic_t=antip)
    v = synth.spinor(dims, 8)
    F = eigenvalue_force(op, v)
    assert np.max(np.abs(F - np.conj(np.swapaxes(F, -1, -2)))) < 1e-15
    assert np.max(np.abs(np.trace(F, axis1=-2, axis2=-1))) < 1e-15
    for X in synth.su3_directions(dims, 9, 2):
        con = np.sum(X * np.swapaxes(F, -1, -2))
        ref = eigenvalue_derivative(op, X, v)
        assert abs(con.imag) < 1e-14 and abs(con.real - ref) < 1e-12 * abs(ref)


def test_force_single_link_central_difference():
    """One link moved alone: tr(X F) at that link against the central
    difference of the Rayleigh quotient v^H Q(U(+-h)) v / v^H v (h = 1e-5),
    for a time link across the antiperiodic boundary and a spatial link."""
    from oracle.dirac import eigenvalue_force
    dims = (4, 2, 2, 2)
    U = synth.gauge_field(dims, 0.5, 17)
    op = WilsonClover(U, -0.3, 1.5)
    v = synth.spinor(dims, 18)
    F = eigenvalue_force(op, v)
    Xall = synth.su3_directions(dims, 19, 1)[0]
    h = 1e-5
    for site, mu in [((3, 1, 0, 1), 0), ((1, 0, 1, 1), 2)]:
        X = np.zeros_like(Xall)
        X[site + (mu,)] = Xall[site + (mu,)]

        def rq(eps):
            Q = WilsonClover(_moved_links(U, X, eps), -0.3, 1.5).Q(v)
            return np.real(np.vdot(v, Q)) / np.real(np.vdot(v, v))
        fd = (rq(h) - rq(-h)) / (2 * h)
        got = np.real(np.trace(X[site + (mu,)] @ F[site + (mu,)]))
        assert abs(got - fd) < 1e-8 * max(abs(fd), 1e-3), (site, mu, got, fd)


@pytest.mark.parametrize("dims,antip,csw", [((2, 2, 2, 2), True, 1.5), ((4, 2, 2, 4), True, 1.5),
                                            ((2, 4, 2, 2), False, 0.0), ((4, 4, 2, 2), False, 1.2)])
def test_bilinear_force_contracts_to_directional_derivative(dims, antip, csw):
    """Force of Re <g, Q psi> for distinct random g, psi: sum tr(X F) equals
    Re <g, Gamma5 (dD/deps) psi> of the product-rule tangent (pinned by
    central differences above); F is traceless Hermitian."""
    from oracle.dirac import bilinear_force, operator_tangent
    U = synth.gauge_field(dims, 0.5, 27)
    op = WilsonClover(U, -0.3, csw, antiperiodic_t=antip)
    g = synth.spinor(dims, 28)
    psi = synth.spinor(dims, 29)
    F = bilinear_force(op, g, psi)
    assert np.max(np.abs(F - np.conj(np.swapaxes(F, -1, -2)))) < 1e-14
    assert np.max(np.abs(np.trace(F, axis1=-2, axis2=-1))) < 1e-14
    for X in synth.su3_directions(dims, 30, 2):
        con = np.sum(X * np.swapaxes(F, -1, -2))
        ref = np.real(np.vdot(g, WilsonClover.g5(operator_tangent(op, X)(psi))))
        assert abs(con.imag) < 1e-13 and abs(con.real - ref) < 1e-12 * abs(ref)


def test_bilinear_force_single_link_central_difference():
    """One link moved alone: tr(X F) against the central difference of
    Re <g, Q(U(+-h)) psi> (h = 1e-5), across the antiperiodic boundary and on a
    spatial link; and the diagonal case g = psi is v^H v times the eigenvalue
    force."""
    from oracle.dirac import bilinear_force, eigenvalue_force
    dims = (4, 2, 2, 2)
    U = synth.gauge_field(dims, 0.5, 37)
    op = WilsonClover(U, -0.3, 1.5)
    g = synth.spinor(dims, 38)
    psi = synth.spinor(dims, 39)
    F = bilinear_force(op, g, psi)
    Xall = synth.su3_directions(dims, 40, 1)[0]
    h = 1e-5
    for site, mu in [((3, 1, 0, 1), 0), ((1, 0, 1, 1), 2)]:
        X = np.zeros_like(Xall)
        X[site + (mu,)] = Xall[site + (mu,)]

        def bl(eps):
            return np.real(np.vdot(g, WilsonClover(_moved_links(U, X, eps), -0.3, 1.5).Q(psi)))
        fd = (bl(h) - bl(-h)) / (2 * h)
        got = np.real(np.trace(X[site + (mu,)] @ F[site + (mu,)]))
        assert abs(got - fd) < 1e-8 * max(abs(fd), 1e-3), (site, mu, got, fd)
    Fd = bilinear_force(op, psi, psi)
    assert np.max(np.abs(Fd - np.real(np.vdot(psi, psi)) * eigenvalue_force(op, psi))) < 1e-12 * np.max(np.abs(Fd))
