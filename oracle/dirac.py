"""Wilson-clover Dirac operator D, Gamma5 and Q = Gamma5 D in plain FP64 numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring): the oracle the GPU
library is checked against.

Conventions (Sec. 2 of the paper, with the readings it leaves open):

* Lattice ``dims = (L0, L1, L2, L3)``; direction mu = 0 is time, the site
  index is lexicographic with mu = 3 fastest.  Fields are numpy arrays with
  the four lattice axes first:
  spinor ``psi[L0, L1, L2, L3, 4 spins, 3 colours]`` (complex128; the
  operators also accept a leading batch axis),
  links ``U[L0, L1, L2, L3, 4 mu, 3, 3]`` with ``U[..., mu, :, :] = U_mu(x)``.
* Lattice spacing a = 1 (Eq. 2.5 writes a; Table 1 quotes a*m0).
* gamma matrices: the paper fixes only the Clifford relations (Eq. 2.3),
  gamma5 = gamma0 gamma1 gamma2 gamma3 (Eq. 2.4) and the representation with
  gamma5 = diag(I2, -I2) (Sec. 2, below Eq. 2.5).  Reading taken: the chiral
  basis gamma0 = -[[0, I2], [I2, 0]], gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]
  (k = 1, 2, 3; sigma_k the Pauli matrices).
* Boundary: the paper says periodic (Sec. 2, below Eq. 2.5); the workloads
  use antiperiodic time.  A hop that crosses the time boundary picks up a
  factor -1 (both directions) when ``antiperiodic_t`` is set; links are not
  modified, so the clover term never sees the phase.
* Clover (Sec. 4, "clover improved ... block diagonal term with 6x6 diagonal
  blocks"; Sheikholeslami-Wohlert).  Reading taken:
  D += c_sw * (i/4) * sum_{mu,nu} sigma_{mu nu} (x) F_{mu nu}(x),
  sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu],
  F_{mu nu} = (1/8) (Q_{mu nu} - Q_{mu nu}^H) with Q_{mu nu}(x) the sum of the
  four plaquette leaves in the (mu, nu) plane that start and end at x.
  No trace is subtracted from F.
"""
import numpy as np

# ---------------------------------------------------------------- gamma basis
_I2 = np.eye(2, dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)
_PAULI = (
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
)


def gamma_matrices():
    """The four Hermitian gamma matrices (Eq. 2.3) and gamma5 (Eq. 2.4).

    Returns ``(g, g5)`` with ``g`` of shape (4, 4, 4): g[mu] = gamma_mu, and
    g5 = g[0] g[1] g[2] g[3], which in this basis is diag(1, 1, -1, -1).
    """
    g = np.empty((4, 4, 4), dtype=np.complex128)
    g[0] = -np.block([[_Z2, _I2], [_I2, _Z2]])
    for k in range(3):
        g[k + 1] = np.block([[_Z2, -1j * _PAULI[k]], [1j * _PAULI[k], _Z2]])
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g, g5


GAMMA, GAMMA5 = gamma_matrices()


def sigma_munu(mu, nu):
    """sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu] (clover term, reading above)."""
    return 0.5j * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])


# ---------------------------------------------------------------- geometry
def volume(dims):
    return int(np.prod(dims))


def shift_field(f, mu, sign):
    """f(x + sign * mu_hat) with periodic wrap (no boundary phase)."""
    return np.roll(f, -sign, axis=mu)


def hop_spinor(psi, mu, sign, antiperiodic_t):
    """psi(x + sign*mu_hat) including the fermion boundary phase of the time
    direction (reading: -1 on hops across t = L0-1 <-> 0 when antiperiodic).
    ``psi`` has shape (..., L0, L1, L2, L3, 4, 3)."""
    out = np.roll(psi, -sign, axis=mu - 6)
    if mu == 0 and antiperiodic_t:
        L0 = psi.shape[-6]
        edge = (Ellipsis, L0 - 1 if sign > 0 else 0) + (slice(None),) * 5
        out[edge] *= -1.0   # x at the last (first) time slice reads across the boundary
    return out


def _dag(M):
    return np.conj(np.swapaxes(M, -1, -2))


def _cmul(U, psi):
    """Colour matrix (..., 3, 3) times spinor (..., 4, 3) on the colour index:
    out[s, a] = sum_b U[a, b] psi[s, b] (as a batched matrix product psi U^T)."""
    return np.matmul(psi, np.swapaxes(U, -1, -2))


def _smul(G, psi):
    """Spin matrix (4, 4) times spinor (..., 4, 3) on the spin index:
    out[s, c] = sum_t G[s, t] psi[t, c]."""
    return np.matmul(G, psi)


# ---------------------------------------------------------------- clover
def plaquette_leaves(U, mu, nu):
    """Q_{mu nu}(x): sum of the four plaquette leaves in the (mu, nu) plane
    starting and ending at x, all with the same orientation (clover term)."""
    Umu = U[..., mu, :, :]
    Unu = U[..., nu, :, :]
    S = shift_field
    Umu_m = S(Umu, mu, -1)            # U_mu(x - mu)
    Unu_m = S(Unu, nu, -1)            # U_nu(x - nu)
    leaf1 = Umu @ S(Unu, mu, +1) @ _dag(S(Umu, nu, +1)) @ _dag(Unu)
    leaf2 = Unu @ _dag(S(S(Umu, nu, +1), mu, -1)) @ _dag(S(Unu, mu, -1)) @ Umu_m
    leaf3 = _dag(Umu_m) @ _dag(S(S(Unu, mu, -1), nu, -1)) @ S(S(Umu, mu, -1), nu, -1) @ Unu_m
    leaf4 = _dag(Unu_m) @ S(Umu, nu, -1) @ S(S(Unu, mu, +1), nu, -1) @ _dag(Umu)
    return leaf1 + leaf2 + leaf3 + leaf4


def field_strength(U, mu, nu):
    """F_{mu nu}(x) = (Q_{mu nu} - Q_{mu nu}^H) / 8 (clover reading, module header)."""
    Q = plaquette_leaves(U, mu, nu)
    return (Q - _dag(Q)) / 8.0


def clover_field(U, csw):
    """Site-diagonal clover matrices as full 12x12 blocks, index s*3 + c.

    C(x) = c_sw * (i/4) * sum_{mu != nu} sigma_{mu nu} (x) F_{mu nu}(x)
         = c_sw * (i/2) * sum_{mu < nu} sigma_{mu nu} (x) F_{mu nu}(x).
    Returns an array of shape dims + (12, 12).
    """
    dims = U.shape[:4]
    C = np.zeros(dims + (12, 12), dtype=np.complex128)
    if csw == 0.0:
        return C
    for mu in range(4):
        for nu in range(mu + 1, 4):
            F = field_strength(U, mu, nu)
            C += np.einsum('st,...ab->...satb', sigma_munu(mu, nu), F).reshape(dims + (12, 12))
    return C * (csw * 0.5j)


# ---------------------------------------------------------------- operators
class WilsonClover:
    """The operator D of Eq. 2.5 (a = 1) plus the clover term.

    (D psi)(x) = (m0 + 4) psi(x) + C(x) psi(x)
                 - 1/2 sum_mu (I4 - gamma_mu) (x) U_mu(x) psi(x + mu)
                 - 1/2 sum_mu (I4 + gamma_mu) (x) U_mu(x - mu)^H psi(x - mu)
    """

    def __init__(self, U, m0, csw, antiperiodic_t=True):
        self.U = np.asarray(U, dtype=np.complex128)
        self.dims = tuple(self.U.shape[:4])
        self.m0 = float(m0)
        self.csw = float(csw)
        self.antiperiodic_t = bool(antiperiodic_t)
        self.C = clover_field(self.U, self.csw)
        self.Ub = [shift_field(self.U[..., mu, :, :], mu, -1) for mu in range(4)]  # U_mu(x-mu)
        self.n = volume(self.dims) * 12

    # ---- pieces of Eq. 2.5
    def diag(self, psi):
        """(m0 + 4) psi + C psi: the site-diagonal part."""
        Cpsi = np.einsum('...ij,...j->...i', self.C,
                         psi.reshape(psi.shape[:-2] + (12,))).reshape(psi.shape)
        return (self.m0 + 4.0) * psi + Cpsi

    def hop(self, psi, mu, sign):
        """The hop term of direction sign*mu of Eq. 2.5 (including -1/2):
        sign=+1: -1/2 (I - gamma_mu) (x) U_mu(x) psi(x + mu)
        sign=-1: -1/2 (I + gamma_mu) (x) U_mu(x - mu)^H psi(x - mu)."""
        nb = hop_spinor(psi, mu, sign, self.antiperiodic_t)
        if sign > 0:
            Up = _cmul(self.U[..., mu, :, :], nb)
            return -0.5 * (Up - _smul(GAMMA[mu], Up))
        Up = _cmul(_dag(self.Ub[mu]), nb)
        return -0.5 * (Up + _smul(GAMMA[mu], Up))

    def D(self, psi):
        out = self.diag(psi)
        for mu in range(4):
            out = out + self.hop(psi, mu, +1) + self.hop(psi, mu, -1)
        return out

    @staticmethod
    def g5(psi):
        """Gamma5 = I (x) gamma5 (x) I3 (Sec. 2, above Eq. 2.7)."""
        return _smul(GAMMA5, psi)

    def Q(self, psi):
        """Q = Gamma5 D (Sec. 2, definition of the Hermitian Wilson-Dirac operator)."""
        return self.g5(self.D(psi))

    def Q_shift(self, psi, tau):
        """(Q - tau I) psi: the shifted operator of Eq. 1.1 / Eq. 3.6."""
        return self.Q(psi) - tau * psi

    def D_g5shift(self, psi, tau):
        """(D - tau Gamma5) psi: the Gamma5-preconditioned operator of Eq. 3.7."""
        return self.D(psi) - tau * self.g5(psi)

    # ---- flat views, [site][spin][colour] order
    def shape_field(self, v):
        return np.asarray(v, dtype=np.complex128).reshape(self.dims + (4, 3))

    def dense(self, which='Q', tau=0.0, chunk=384):
        """Dense matrix of Q - tau, D - tau*Gamma5 or D by applying the operator
        to every unit vector (brute force, small lattices only)."""
        n = self.n
        M = np.empty((n, n), dtype=np.complex128)
        for j0 in range(0, n, chunk):
            j1 = min(n, j0 + chunk)
            E = np.zeros((j1 - j0, n), dtype=np.complex128)
            E[np.arange(j1 - j0), np.arange(j0, j1)] = 1.0
            psi = E.reshape((j1 - j0,) + self.dims + (4, 3))
            if which == 'Q':
                col = self.Q_shift(psi, tau)
            elif which == 'Dg5':
                col = self.D_g5shift(psi, tau)
            else:
                col = self.D(psi)
            M[:, j0:j1] = col.reshape(j1 - j0, n).T
        return M


def clover_blocks(C):
    """The two 6x6 chirality blocks of each 12x12 clover matrix: block 0 is
    spins {0, 1} (gamma5 = +1), block 1 spins {2, 3}.  Returns (..., 2, 6, 6)."""
    out = np.empty(C.shape[:-2] + (2, 6, 6), dtype=np.complex128)
    out[..., 0, :, :] = C[..., :6, :6]
    out[..., 1, :, :] = C[..., 6:, 6:]
    return out


# ---------------------------------------------------------------- derivative along a link direction
# The eigenvalue derivative of the differentiation workload: links move as
# U_mu(x) -> exp(i eps X_mu(x)) U_mu(x) with X traceless Hermitian, so
# dU/deps at eps = 0 is i X U.  The operator of Eq. 2.5 plus the clover term is
# linear in each link of the hop terms and a sum of four-link products in the
# clover leaves; its derivative follows by the product rule.  For a simple
# eigenvalue lambda of the Hermitian Q with unit eigenvector v,
# d lambda / d eps = v^H (dQ/d eps) v (Hellmann-Feynman).

def _dag_pair(p):
    return _dag(p[0]), _dag(p[1])


def _shift_pair(p, mu, sign):
    return shift_field(p[0], mu, sign), shift_field(p[1], mu, sign)


def _product_rule(pairs):
    """(A1 A2 ... Ak, d(A1 A2 ... Ak)) from (Ai, dAi) pairs."""
    P, dP = pairs[0]
    for M, dM in pairs[1:]:
        dP = dP @ M + P @ dM
        P = P @ M
    return P, dP


def plaquette_leaves_tangent(U, dU, mu, nu):
    """d Q_{mu nu}(x) along dU: the four leaves of ``plaquette_leaves``
    differentiated factor by factor."""
    Umu = (U[..., mu, :, :], dU[..., mu, :, :])
    Unu = (U[..., nu, :, :], dU[..., nu, :, :])
    S = _shift_pair
    D = _dag_pair
    Umu_m = S(Umu, mu, -1)
    Unu_m = S(Unu, nu, -1)
    leaves = [
        [Umu, S(Unu, mu, +1), D(S(Umu, nu, +1)), D(Unu)],
        [Unu, D(S(S(Umu, nu, +1), mu, -1)), D(S(Unu, mu, -1)), Umu_m],
        [D(Umu_m), D(S(S(Unu, mu, -1), nu, -1)), S(S(Umu, mu, -1), nu, -1), Unu_m],
        [D(Unu_m), S(Umu, nu, -1), S(S(Unu, mu, +1), nu, -1), D(Umu)],
    ]
    return sum(_product_rule(l)[1] for l in leaves)


def clover_field_tangent(U, dU, csw):
    """dC/deps of ``clover_field`` along dU (dims + (12, 12))."""
    dims = U.shape[:4]
    dC = np.zeros(dims + (12, 12), dtype=np.complex128)
    if csw == 0.0:
        return dC
    for mu in range(4):
        for nu in range(mu + 1, 4):
            dQ = plaquette_leaves_tangent(U, dU, mu, nu)
            dF = (dQ - _dag(dQ)) / 8.0
            dC += np.einsum('st,...ab->...satb', sigma_munu(mu, nu), dF).reshape(dims + (12, 12))
    return dC * (csw * 0.5j)


def link_tangent(U, X):
    """dU/deps = i X U for U_mu(x) -> exp(i eps X_mu(x)) U_mu(x)."""
    return 1j * np.einsum('...ab,...bc->...ac', X, U)


def operator_tangent(op, X):
    """Callable psi -> (dD/deps) psi for the WilsonClover ``op`` along X: the
    hop terms of Eq. 2.5 with dU in place of U (the (m0 + 4) term is constant)
    plus the clover derivative."""
    dU = link_tangent(op.U, X)
    dC = clover_field_tangent(op.U, dU, op.csw)
    dUb = [shift_field(dU[..., mu, :, :], mu, -1) for mu in range(4)]

    def apply(psi):
        out = np.einsum('...ij,...j->...i', dC, psi.reshape(psi.shape[:-2] + (12,))).reshape(psi.shape)
        for mu in range(4):
            nb = hop_spinor(psi, mu, +1, op.antiperiodic_t)
            Up = _cmul(dU[..., mu, :, :], nb)
            out = out - 0.5 * (Up - _smul(GAMMA[mu], Up))
            nb = hop_spinor(psi, mu, -1, op.antiperiodic_t)
            Up = _cmul(_dag(dUb[mu]), nb)
            out = out - 0.5 * (Up + _smul(GAMMA[mu], Up))
        return out
    return apply


def eigenvalue_derivative(op, X, v):
    """Hellmann-Feynman d lambda / d eps = Re v^H Gamma5 (dD/deps) v for a unit
    eigenvector v of Q = Gamma5 D with a simple eigenvalue."""
    v = np.asarray(v).reshape(op.dims + (4, 3))
    dv = operator_tangent(op, X)(v)
    return float(np.real(np.vdot(v, WilsonClover.g5(dv))) / np.real(np.vdot(v, v)))


# ---------------------------------------------------------------- force: the derivative per link
# The same derivative resolved link by link: a traceless Hermitian 3x3 matrix
# F_mu(x) per link with d lambda / d eps = sum_{x, mu} tr(X_mu(x) F_mu(x)) for
# every traceless Hermitian direction field X.  With w = Gamma5 v:
#
# * hop terms of Eq. 2.5: the backward hop is the complex conjugate of the
#   forward one (Q is Hermitian), so both together give -Re tr(dU_mu(x) A_mu(x))
#   with the colour outer product A = sum_{st} (I - gamma_mu)_{st}
#   v_t(x + mu) w_s(x)^H (boundary phase included in v(x + mu));
# * clover term: v^H Gamma5 C v is real, so its derivative is
#   Re[i c_sw / 16 * sum_x sum_{(rho, nu) ordered} tr(dQ_{rho nu}(x) Bt(x))] with
#   Bt = B + B^H, B = sum_{st} sigma_{rho nu, st} v_t(x) w_s(x)^H; a link U_rho(y)
#   sits in the plaquette above it (non-daggered, corner y at the lower left) and
#   in the one below it (daggered) of each plane (rho, nu), and each plaquette
#   is a leaf at each of its four corners.


def _traceless_hermitian(K):
    H = 0.5 * (K + _dag(K))
    tr = np.trace(H, axis1=-2, axis2=-1)
    return H - tr[..., None, None] * np.eye(3) / 3.0


def eigenvalue_force(op, v):
    """F_mu(x) (dims + (4, 3, 3)), traceless Hermitian, such that
    d lambda / d eps = sum tr(X_mu(x) F_mu(x)) / (v^H v) along any traceless
    Hermitian X (links moving as exp(i eps X) U); v a unit-norm-free eigenvector
    of Q with a simple eigenvalue (Hellmann-Feynman, resolved per link)."""
    v = np.asarray(v).reshape(op.dims + (4, 3))
    w = WilsonClover.g5(v)
    wc = np.conj(w)
    U = op.U
    S = shift_field
    K = np.zeros(op.dims + (4, 3, 3), dtype=np.complex128)
    I4 = np.eye(4, dtype=np.complex128)
    for rho in range(4):
        nb = hop_spinor(v, rho, +1, op.antiperiodic_t)
        A = np.einsum('st,...ta,...sb->...ab', I4 - GAMMA[rho], nb, wc)
        K[..., rho, :, :] -= 1j * (U[..., rho, :, :] @ A)
    if op.csw != 0.0:
        c = op.csw / 16.0
        for rho in range(4):
            for nu in range(4):
                if nu == rho:
                    continue
                B = np.einsum('st,...ta,...sb->...ab', sigma_munu(rho, nu), v, wc)
                Bt = B + _dag(B)
                Ur = U[..., rho, :, :]
                Un = U[..., nu, :, :]
                # plaquette above U_rho(y): a b c d from y, corners y, y+rho, y+rho+nu, y+nu
                a = Ur
                b = S(Un, rho, +1)
                cc = _dag(S(Ur, nu, +1))
                d = _dag(Un)
                B0, B1 = Bt, S(Bt, rho, +1)
                B2, B3 = S(S(Bt, rho, +1), nu, +1), S(Bt, nu, +1)
                above = (a @ b @ cc @ d @ B0 + a @ B1 @ b @ cc @ d
                         + a @ b @ B2 @ cc @ d + a @ b @ cc @ B3 @ d)
                # plaquette below U_rho(y): path y -> y-nu -> y-nu+rho -> y+rho, then U_rho(y)^H
                dp = _dag(S(Un, nu, -1))
                ap = S(Ur, nu, -1)
                bp = S(S(Un, rho, +1), nu, -1)
                C0, C1 = Bt, S(Bt, nu, -1)
                C2, C3 = S(S(Bt, nu, -1), rho, +1), S(Bt, rho, +1)
                below = (C0 @ dp @ ap @ bp + dp @ C1 @ ap @ bp
                         + dp @ ap @ C2 @ bp + dp @ ap @ bp @ C3) @ _dag(Ur)
                K[..., rho, :, :] += c * below - c * above
    return _traceless_hermitian(K) / float(np.real(np.vdot(v, v)))


def bilinear_force(op, g, psi):
    """Per-link force of the real bilinear form Re <g, Q psi> (the link
    gradient of a real loss through psi -> Q psi with cotangent g): F_mu(x)
    (dims + (4, 3, 3)), traceless Hermitian, such that
    d/d eps Re <g, Q(U(eps)) psi> = sum tr(X_mu(x) F_mu(x)) for links moving
    as exp(i eps X) U.  Restates ``eigenvalue_force`` for two vectors:

    * hop terms: Q' is Hermitian, so the backward hop of <g, Q' psi> is the
      complex conjugate of the forward hop of <psi, Q' g>; the real part is
      the sum of the real parts of the two forward terms, and the force is
      -i U (A(psi, g) + A(g, psi)) / 2 with A(a, b) = sum_{st}
      (I - gamma_mu)_{st} a_t(x + mu) (Gamma5 b)_s(x)^H;
    * clover term: as in ``eigenvalue_force`` with B = sum_{st} sigma_st
      psi_t(x) (Gamma5 g)_s(x)^H (the real part of the derivative again needs
      only Bt = B + B^H).

    For g = psi = v this is v^H v times ``eigenvalue_force(op, v)``."""
    g = np.asarray(g).reshape(op.dims + (4, 3))
    psi = np.asarray(psi).reshape(op.dims + (4, 3))
    wg = np.conj(WilsonClover.g5(g))
    wp = np.conj(WilsonClover.g5(psi))
    U = op.U
    S = shift_field
    K = np.zeros(op.dims + (4, 3, 3), dtype=np.complex128)
    I4 = np.eye(4, dtype=np.complex128)
    for rho in range(4):
        nb_p = hop_spinor(psi, rho, +1, op.antiperiodic_t)
        nb_g = hop_spinor(g, rho, +1, op.antiperiodic_t)
        A = (np.einsum('st,...ta,...sb->...ab', I4 - GAMMA[rho], nb_p, wg)
             + np.einsum('st,...ta,...sb->...ab', I4 - GAMMA[rho], nb_g, wp))
        K[..., rho, :, :] -= 0.5j * (U[..., rho, :, :] @ A)
    if op.csw != 0.0:
        c = op.csw / 16.0
        for rho in range(4):
            for nu in range(4):
                if nu == rho:
                    continue
                B = np.einsum('st,...ta,...sb->...ab', sigma_munu(rho, nu), psi, wg)
                Bt = B + _dag(B)
                Ur = U[..., rho, :, :]
                Un = U[..., nu, :, :]
                a = Ur
                b = S(Un, rho, +1)
                cc = _dag(S(Ur, nu, +1))
                d = _dag(Un)
                B0, B1 = Bt, S(Bt, rho, +1)
                B2, B3 = S(S(Bt, rho, +1), nu, +1), S(Bt, nu, +1)
                above = (a @ b @ cc @ d @ B0 + a @ B1 @ b @ cc @ d
                         + a @ b @ B2 @ cc @ d + a @ b @ cc @ B3 @ d)
                dp = _dag(S(Un, nu, -1))
                ap = S(Ur, nu, -1)
                bp = S(S(Un, rho, +1), nu, -1)
                C0, C1 = Bt, S(Bt, nu, -1)
                C2, C3 = S(S(Bt, nu, -1), rho, +1), S(Bt, rho, +1)
                below = (C0 @ dp @ ap @ bp + dp @ C1 @ ap @ bp
                         + dp @ ap @ C2 @ bp + dp @ ap @ bp @ C3) @ _dag(Ur)
                K[..., rho, :, :] += c * below - c * above
    return _traceless_hermitian(K)
