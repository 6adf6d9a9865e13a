"""Aggregation multigrid for the shifted Wilson-clover systems, plain FP64 numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

What is restated here (Sec. 2 "Algebraic multigrid methods", Sec. 3 "Local
coherence", Sec. 4 "Solving the correction equation" and Table 2):

* aggregation interpolation P built from test vectors, split by chirality so
  that Gamma5 P = P Gamma5^c (Sec. 2, text above Eq. 2.9; Fig. "buildP");
* restriction R = P^H and the Galerkin coarse operator D_c = P^H D P,
  Q_c = Gamma5^c D_c (Sec. 2, Eq. 2.8 and Eq. 2.9), kept as a nearest-
  neighbour block stencil on the coarse lattice;
* the SAP smoother, red-black multiplicative Schwarz over lattice blocks
  with approximate GMRES block solves (Eq. 2.10, Proposition 1, Sec. 4
  "Impact of the smoother");
* GMRES, flexible GMRES and the two-level cycle E_2g with post-smoothing only
  (Eq. 2.8, Table 2);
* the adaptive setup of the test vectors (Table 2; the procedure itself is
  deferred by the paper to the DD-alpha-AMG literature -- reading below);
* the three-level hierarchy: the aggregation and Galerkin construction
  applied to the coarse operator, and the K-cycle whose middle level is
  FGMRES preconditioned by the level-1 two-level cycle (``ThreeLevelMG``;
  readings in its docstring).

Readings taken where the paper is silent:

* Coarse degrees of freedom per coarse site are ordered [chirality][i < N_v];
  chirality 0 collects spins {0, 1} (gamma5 = +1), chirality 1 spins {2, 3}.
  Gamma5^c = diag(+1 x N_v, -1 x N_v).
* Each aggregate's N_v restricted test vectors are orthonormalised by
  modified Gram-Schmidt applied twice.
* Coarse stencil directions d: 0 = self, 1 + mu = +mu, 5 + mu = -mu.
  A fine hop is attributed to direction +-mu when it leaves the lattice block
  (and the coarse extent in mu is > 1), else to the self term.
* SAP: block colour = (sum of block coordinates) mod 2, colour 0 first; the
  block operator drops the hops that leave the block (Dirichlet cut); every
  block-grid extent must be even so that blocks of one colour never touch.
* The cycle is E_2g with mu = 0 pre- and nu post-smoothing steps (Table 2
  lists "(post-)smoothing steps"); one SAP "step" is one red+black sweep.
* Setup: iteration 1 smooths each random test vector on D x = 0; later
  iterations replace each vector by one application of the current
  two-level preconditioner to it (inverse iteration); P and D_c are rebuilt
  after every iteration.  Its result is not unique (only the solver's speed
  depends on it) and the GPU setup is not compared with it; it is pinned by
  a property only: the vectors it returns approach the near-kernel of D.
"""
import numpy as np

from .dirac import GAMMA5


# ----------------------------------------------------------------- geometry
class Blocking:
    """A partition of the lattice ``dims`` into blocks of extent ``block``.

    ``sites[b, l]`` is the flat fine-site index of local site ``l`` of block
    ``b``; blocks and local sites are both lexicographic with mu = 3 fastest.
    """

    def __init__(self, dims, block):
        dims = tuple(int(d) for d in dims)
        block = tuple(int(b) for b in block)
        for L, b in zip(dims, block):
            if b <= 0 or L % b:
                raise ValueError(f"block {block} does not divide lattice {dims}")
        self.dims, self.block = dims, block
        self.cdims = tuple(L // b for L, b in zip(dims, block))
        self.nblocks = int(np.prod(self.cdims))
        self.bsites = int(np.prod(block))
        c = np.indices(self.cdims).reshape(4, -1).T           # block coords (nb, 4)
        l = np.indices(block).reshape(4, -1).T                # local coords (bs, 4)
        x = c[:, None, :] * np.array(block) + l[None, :, :]   # fine coords
        self.sites = np.ravel_multi_index(tuple(np.moveaxis(x, -1, 0)), dims)
        self.colour = c.sum(axis=1) % 2
        self.bcoords = c

    def _split_shape(self):
        sh = []
        for c, b in zip(self.cdims, self.block):
            sh += [c, b]
        return tuple(sh)

    def gather(self, f, tail):
        """dims + tail -> (nblocks, bsites) + tail, the same as
        ``f.reshape((-1,) + tail)[self.sites]`` (a pure re-indexing: each fine
        axis split into (block coordinate, local coordinate), block axes
        first)."""
        nt = len(tail)
        g = np.asarray(f).reshape(self._split_shape() + tail)
        g = g.transpose((0, 2, 4, 6, 1, 3, 5, 7) + tuple(range(8, 8 + nt)))
        return g.reshape((self.nblocks, self.bsites) + tail)

    def scatter(self, fb, tail):
        """(nblocks, bsites) + tail -> dims + tail (inverse of ``gather``)."""
        nt = len(tail)
        g = np.asarray(fb).reshape(tuple(self.cdims) + tuple(self.block) + tail)
        g = g.transpose((0, 4, 1, 5, 2, 6, 3, 7) + tuple(range(8, 8 + nt)))
        return np.ascontiguousarray(g).reshape(self.dims + tail)


def _flat(psi):
    return psi.reshape((-1, 4, 3))


# ----------------------------------------------------------------- GMRES
def gmres(apply, b, tol, maxiter, dot=None):
    """GMRES with zero initial guess (Saad), run independently on a batch of
    systems ``b`` of shape (nb, n); Arnoldi by modified Gram-Schmidt, complex
    Givens rotations.  System k stops once its residual estimate is
    <= tol * ||b_k|| or after ``maxiter`` steps.

    Returns ``(x, iters)``.
    """
    if dot is None:
        def dot(u, v):
            return np.einsum('bi,bi->b', np.conj(u), v)
    b = np.asarray(b)
    nb, n = b.shape
    m = int(maxiter)
    beta = np.sqrt(np.maximum(dot(b, b).real, 0.0))
    Vk = np.zeros((m + 1, nb, n), dtype=np.complex128)
    H = np.zeros((nb, m + 1, m), dtype=np.complex128)
    cs = np.zeros((nb, m), dtype=np.float64)
    sn = np.zeros((nb, m), dtype=np.complex128)
    g = np.zeros((nb, m + 1), dtype=np.complex128)
    g[:, 0] = beta
    safe = np.where(beta > 0, beta, 1.0)
    Vk[0] = b / safe[:, None]
    active = beta > 0
    k = np.zeros(nb, dtype=np.int64)
    for j in range(m):
        if not active.any():
            break
        w = apply(Vk[j])
        w = np.where(active[:, None], w, 0.0)
        for i in range(j + 1):
            h = dot(Vk[i], w)
            H[:, i, j] = h
            w = w - h[:, None] * Vk[i]
        hn = np.sqrt(np.maximum(dot(w, w).real, 0.0))
        H[:, j + 1, j] = hn
        Vk[j + 1] = np.where((hn > 0)[:, None], w / np.where(hn > 0, hn, 1.0)[:, None], 0.0)
        for i in range(j):
            a = H[:, i, j].copy()
            c = H[:, i + 1, j].copy()
            H[:, i, j] = cs[:, i] * a + sn[:, i] * c
            H[:, i + 1, j] = -np.conj(sn[:, i]) * a + cs[:, i] * c
        a = H[:, j, j].copy()
        c = H[:, j + 1, j].copy()
        r = np.sqrt(np.abs(a) ** 2 + np.abs(c) ** 2)
        absa = np.abs(a)
        rs = np.where(r > 0, r, 1.0)
        cs[:, j] = np.where(absa > 0, absa / rs, 0.0)
        sn[:, j] = np.where(absa > 0, (a / np.where(absa > 0, absa, 1.0)) * np.conj(c) / rs,
                            1.0 + 0j)
        H[:, j, j] = cs[:, j] * a + sn[:, j] * c
        H[:, j + 1, j] = 0.0
        g[:, j + 1] = -np.conj(sn[:, j]) * g[:, j]
        g[:, j] = cs[:, j] * g[:, j]
        k = np.where(active, j + 1, k)
        done = np.abs(g[:, j + 1]) <= tol * beta
        active = active & ~done
    x = np.zeros((nb, n), dtype=np.complex128)
    for s in range(nb):
        ks = int(k[s])
        if ks == 0:
            continue
        y = _backsolve(H[s, :ks, :ks], g[s, :ks])
        x[s] = np.tensordot(y, Vk[:ks, s, :], axes=(0, 0))
    return x, k


def _backsolve(R, g):
    n = R.shape[0]
    y = np.zeros(n, dtype=np.complex128)
    for i in range(n - 1, -1, -1):
        y[i] = (g[i] - R[i, i + 1:] @ y[i + 1:]) / R[i, i] if R[i, i] != 0 else 0.0
    return y


def fgmres(apply, precond, b, tol, maxiter, x0=None):
    """Flexible GMRES (right preconditioning with a varying preconditioner,
    Saad 1993) for one system; Arnoldi by modified Gram-Schmidt.  Stops when
    the residual estimate is <= tol * ||b - A x0|| or after ``maxiter`` steps.

    Returns ``(x, iters, resnorm_estimate)``.
    """
    b = np.asarray(b).reshape(-1)
    n = b.size
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128).reshape(-1)
    r = b - apply(x) if x0 is not None else b.copy()
    beta = np.linalg.norm(r)
    m = int(maxiter)
    if beta == 0:
        return x, 0, 0.0
    Vk = [r / beta]
    Z = []
    H = np.zeros((m + 1, m), dtype=np.complex128)
    cs = np.zeros(m)
    sn = np.zeros(m, dtype=np.complex128)
    g = np.zeros(m + 1, dtype=np.complex128)
    g[0] = beta
    k = 0
    for j in range(m):
        z = precond(Vk[j])
        Z.append(z)
        w = apply(z)
        for i in range(j + 1):
            H[i, j] = np.vdot(Vk[i], w)
            w = w - H[i, j] * Vk[i]
        H[j + 1, j] = np.linalg.norm(w)
        Vk.append(w / H[j + 1, j] if H[j + 1, j] != 0 else w)
        for i in range(j):
            a, c = H[i, j], H[i + 1, j]
            H[i, j] = cs[i] * a + sn[i] * c
            H[i + 1, j] = -np.conj(sn[i]) * a + cs[i] * c
        a, c = H[j, j], H[j + 1, j]
        rr = np.hypot(abs(a), abs(c))
        if abs(a) > 0:
            cs[j] = abs(a) / rr
            sn[j] = (a / abs(a)) * np.conj(c) / rr
        else:
            cs[j], sn[j] = 0.0, 1.0
        H[j, j] = cs[j] * a + sn[j] * c
        H[j + 1, j] = 0.0
        g[j + 1] = -np.conj(sn[j]) * g[j]
        g[j] = cs[j] * g[j]
        k = j + 1
        if abs(g[j + 1]) <= tol * beta:
            break
    y = _backsolve(H[:k, :k], g[:k])
    for i in range(k):
        x = x + y[i] * Z[i]
    return x, k, float(abs(g[k]))


# ----------------------------------------------------------------- interpolation
class Interpolation:
    """Aggregation-based interpolation with chirality split (Sec. 2, text
    above Eq. 2.9 and Fig. "buildP"; Sec. 3 "Local coherence").

    ``P[b, chi, i, l, s, c]``: coarse site b, chirality chi, vector i, local
    site l, spin s in {2 chi, 2 chi + 1}, colour c.
    """

    def __init__(self, dims, block, vectors):
        self.blk = Blocking(dims, block)
        W = np.asarray(vectors, dtype=np.complex128)
        self.nv = W.shape[0]
        nb, bs = self.blk.nblocks, self.blk.bsites
        Wf = W.reshape(self.nv, -1, 4, 3)[:, self.blk.sites]      # (nv, nb, bs, 4, 3)
        P = np.zeros((nb, 2, self.nv, bs, 2, 3), dtype=np.complex128)
        for chi in range(2):
            Wc = Wf[..., 2 * chi:2 * chi + 2, :].reshape(self.nv, nb, bs * 6)
            Wc = np.transpose(Wc, (1, 0, 2)).copy()                # (nb, nv, bs*6)
            for _ in range(2):                                      # MGS, twice
                for i in range(self.nv):
                    for j in range(i):
                        h = np.einsum('bk,bk->b', np.conj(Wc[:, j]), Wc[:, i])
                        Wc[:, i] -= h[:, None] * Wc[:, j]
                    nrm = np.linalg.norm(Wc[:, i], axis=1)
                    Wc[:, i] /= np.where(nrm > 0, nrm, 1.0)[:, None]
            P[:, chi] = Wc.reshape(nb, self.nv, bs, 2, 3)
        self.P = P
        self.dims = tuple(dims)
        self.nc = 2 * self.nv

    def restrict(self, r):
        """R r = P^H r; returns coarse vector (nblocks, 2, nv) (Eq. 2.8, R = P^H)."""
        rb = self.blk.gather(r, (4, 3))                                 # (nb, bs, 4, 3)
        out = np.empty((self.blk.nblocks, 2, self.nv), dtype=np.complex128)
        nb = self.blk.nblocks
        for chi in range(2):
            # per aggregate: the nv inner products <P_i, r> = conj(sum P_i conj(r))
            # over (site, spin, colour)
            Pc = self.P[:, chi].reshape(nb, self.nv, -1)
            rc = np.conj(rb[:, :, 2 * chi:2 * chi + 2, :]).reshape(nb, -1, 1)
            out[:, chi] = np.conj(np.matmul(Pc, rc)[..., 0])
        return out

    def prolong(self, xc):
        """P x_c as a fine field dims + (4, 3)."""
        xc = np.asarray(xc).reshape(self.blk.nblocks, 2, self.nv)
        fb = np.zeros((self.blk.nblocks, self.blk.bsites, 4, 3), dtype=np.complex128)
        for chi in range(2):
            fb[:, :, 2 * chi:2 * chi + 2, :] = np.einsum('bilsc,bi->blsc', self.P[:, chi], xc[:, chi])
        return self.blk.scatter(fb, (4, 3))

    def dense(self):
        """P as a dense (12 V) x (2 nv nblocks) matrix (small lattices only)."""
        ncol = self.blk.nblocks * self.nc
        M = np.zeros((int(np.prod(self.dims)) * 12, ncol), dtype=np.complex128)
        e = np.zeros(ncol, dtype=np.complex128)
        for j in range(ncol):
            e[j] = 1.0
            M[:, j] = self.prolong(e).reshape(-1)
            e[j] = 0.0
        return M


class CoarseInterpolation:
    """The same aggregation one level down (three-level hierarchy, Sec. 2
    "Algebraic multigrid methods": the construction is applied recursively).
    A level-1 vector x[site, chi, i] (N_v1 components per chirality) is cut
    into level-2 aggregates of extent ``block`` on the level-1 lattice and
    split by the level-1 chirality index, so Gamma5^c P2 = P2 Gamma5^cc; each
    (aggregate, chirality) piece of the test vectors is orthonormalised by
    modified Gram-Schmidt applied twice.

    ``P[b, chi, j, l, i]``: level-2 site b, chirality chi, vector j, local
    level-1 site l, component i < N_v1 of chirality chi.
    """

    def __init__(self, cdims, block, nv_in, vectors):
        self.blk = Blocking(cdims, block)
        self.nv_in = int(nv_in)
        W = np.asarray(vectors, dtype=np.complex128)
        self.nv = W.shape[0]
        nb, bs = self.blk.nblocks, self.blk.bsites
        Wf = W.reshape(self.nv, -1, 2, self.nv_in)[:, self.blk.sites]   # (nv, nb, bs, 2, nv_in)
        P = np.zeros((nb, 2, self.nv, bs, self.nv_in), dtype=np.complex128)
        for chi in range(2):
            Wc = np.transpose(Wf[..., chi, :].reshape(self.nv, nb, bs * self.nv_in), (1, 0, 2)).copy()
            for _ in range(2):
                for i in range(self.nv):
                    for j in range(i):
                        h = np.einsum('bk,bk->b', np.conj(Wc[:, j]), Wc[:, i])
                        Wc[:, i] -= h[:, None] * Wc[:, j]
                    nrm = np.linalg.norm(Wc[:, i], axis=1)
                    Wc[:, i] /= np.where(nrm > 0, nrm, 1.0)[:, None]
            P[:, chi] = Wc.reshape(nb, self.nv, bs, self.nv_in)
        self.P = P
        self.cdims_in = tuple(cdims)
        self.nc = 2 * self.nv

    def restrict(self, r):
        """P2^H r for a level-1 vector r (V1 x 2 N_v1); returns (nb, 2, nv)."""
        rb = np.asarray(r).reshape(-1, 2, self.nv_in)[self.blk.sites]      # (nb, bs, 2, nv_in)
        out = np.empty((self.blk.nblocks, 2, self.nv), dtype=np.complex128)
        for chi in range(2):
            out[:, chi] = np.einsum('bjli,bli->bj', np.conj(self.P[:, chi]), rb[:, :, chi, :])
        return out

    def prolong(self, xc):
        """P2 x_c as a level-1 vector (V1, 2 N_v1)."""
        xc = np.asarray(xc).reshape(self.blk.nblocks, 2, self.nv)
        fb = np.zeros((self.blk.nblocks, self.blk.bsites, 2, self.nv_in), dtype=np.complex128)
        for chi in range(2):
            fb[:, :, chi, :] = np.einsum('bjli,bj->bli', self.P[:, chi], xc[:, chi])
        out = np.zeros((int(np.prod(self.cdims_in)), 2, self.nv_in), dtype=np.complex128)
        out[self.blk.sites.reshape(-1)] = fb.reshape(-1, 2, self.nv_in)
        return out.reshape(-1, 2 * self.nv_in)

    def dense(self):
        ncol = self.blk.nblocks * self.nc
        M = np.zeros((int(np.prod(self.cdims_in)) * 2 * self.nv_in, ncol), dtype=np.complex128)
        e = np.zeros(ncol, dtype=np.complex128)
        for j in range(ncol):
            e[j] = 1.0
            M[:, j] = self.prolong(e).reshape(-1)
            e[j] = 0.0
        return M


def local_coherence(interp, v):
    """Local coherence measure lc(v) = ||Pi v|| / ||v|| (Sec. 3), with Pi the
    orthogonal projection on the range of P: Pi v = P (P^H v), P having
    orthonormal columns (per aggregate and chirality, by construction)."""
    v = np.asarray(v).reshape(interp.dims + (4, 3))
    pv = interp.prolong(interp.restrict(v))
    nv = np.linalg.norm(v)
    return float(np.linalg.norm(pv) / nv) if nv > 0 else 0.0


def gamma5_coarse(nv):
    """Gamma5^c per coarse site: diag(+1 x nv, -1 x nv) (Sec. 2, above Eq. 2.9)."""
    return np.concatenate([np.ones(nv), -np.ones(nv)])


class CoarseOperator:
    """Galerkin coarse operator D_c = P^H D P as a nearest-neighbour stencil
    on the coarse lattice (Eq. 2.8 and Eq. 2.9):

    (D_c x)(b) = sum_{d=0..8} A[b, d] x(b + d),  d: 0 self, 1+mu: +mu, 5+mu: -mu,

    with A[b, d] of size (2 nv) x (2 nv), rows/columns ordered [chi][i].
    """

    def __init__(self, A, cdims, nv):
        self.A = A
        self.cdims = tuple(cdims)
        self.nv = nv
        self.nc = 2 * nv
        self.g5c = gamma5_coarse(nv)

    @classmethod
    def galerkin(cls, op, interp):
        """Build A = P^H D P column class by column class: the fine vector
        v = sum_b P_b e_(chi,i) is pushed through D hop by hop, every hop is
        attributed to the coarse direction it crosses, and the pieces are
        restricted with P^H."""
        blk = interp.blk
        nv, nc = interp.nv, interp.nc
        nb = blk.nblocks
        dims = blk.dims
        A = np.zeros((nb, 9, nc, nc), dtype=np.complex128)
        coords = np.indices(dims)
        face = {}
        for mu in range(4):
            loc = coords[mu] % blk.block[mu]
            leaves = blk.cdims[mu] > 1
            face[(mu, +1)] = (loc == blk.block[mu] - 1) & leaves
            face[(mu, -1)] = (loc == 0) & leaves
        for chi in range(2):
            for i in range(nv):
                e = np.zeros((nb, 2, nv), dtype=np.complex128)
                e[:, chi, i] = 1.0
                v = interp.prolong(e)
                parts = [op.diag(v)] + [np.zeros_like(v) for _ in range(8)]
                for mu in range(4):
                    for sgn, d in ((+1, 1 + mu), (-1, 5 + mu)):
                        h = op.hop(v, mu, sgn)
                        f = face[(mu, sgn)][..., None, None]
                        parts[d] += np.where(f, h, 0.0)
                        parts[0] += np.where(f, 0.0, h)
                col = chi * nv + i
                for d in range(9):
                    A[:, d, :, col] = interp.restrict(parts[d]).reshape(nb, nc)
        return cls(A, blk.cdims, nv)

    @classmethod
    def galerkin_coarse(cls, cop, interp2):
        """The next level's Galerkin operator A2 = P2^H D_c P2 as a stencil on
        the level-2 lattice, built like ``galerkin``: each column class of P2
        goes through the nine terms of the level-1 stencil, and a term that
        reads across the face of a level-2 aggregate (level-2 extent > 1) is
        attributed to that level-2 direction, every other term to the self
        term."""
        blk = interp2.blk
        nv2, nc2, nc1 = interp2.nv, interp2.nc, cop.nc
        nb2 = blk.nblocks
        V1 = int(np.prod(cop.cdims))
        coords = np.indices(blk.dims).reshape(4, -1).T
        face = {}
        for mu in range(4):
            loc = coords[:, mu] % blk.block[mu]
            leaves = blk.cdims[mu] > 1
            face[(mu, +1)] = (loc == blk.block[mu] - 1) & leaves
            face[(mu, -1)] = (loc == 0) & leaves
        A1 = cop.A.reshape(cop.cdims + (9, nc1, nc1))
        A2 = np.zeros((nb2, 9, nc2, nc2), dtype=np.complex128)
        for chi in range(2):
            for j in range(nv2):
                e = np.zeros((nb2, 2, nv2), dtype=np.complex128)
                e[:, chi, j] = 1.0
                v = interp2.prolong(e).reshape(cop.cdims + (nc1,))
                parts = [np.zeros((V1, nc1), dtype=np.complex128) for _ in range(9)]
                for d in range(9):
                    h = np.einsum('...rc,...c->...r', A1[..., d, :, :], cop.neighbour(v, d)).reshape(V1, nc1)
                    if d == 0:
                        parts[0] += h
                        continue
                    f = face[((d - 1) % 4, +1 if d <= 4 else -1)][:, None]
                    parts[d] += np.where(f, h, 0.0)
                    parts[0] += np.where(f, 0.0, h)
                col = chi * nv2 + j
                for d in range(9):
                    A2[:, d, :, col] = interp2.restrict(parts[d]).reshape(nb2, nc2)
        return cls(A2, blk.cdims, nv2)

    def neighbour(self, x, d):
        """x(b + d) on the coarse lattice (periodic; phases live inside A)."""
        if d == 0:
            return x
        mu = (d - 1) % 4
        sgn = +1 if d <= 4 else -1
        return np.roll(x, -sgn, axis=mu)

    def apply_D(self, x):
        """D_c x; x of shape (nblocks, 2 nv) or cdims + (2 nv,)."""
        xs = np.asarray(x).reshape(self.cdims + (self.nc,))
        A = self.A.reshape(self.cdims + (9, self.nc, self.nc))
        y = np.zeros_like(xs)
        for d in range(9):
            y += np.einsum('...rc,...c->...r', A[..., d, :, :], self.neighbour(xs, d))
        return y.reshape(-1, self.nc)

    def apply(self, x, tau, form='g5'):
        """(D_c - tau Gamma5^c) x for form 'g5' (coarse version of Eq. 3.7), or
        (Q_c - tau) x = (Gamma5^c D_c - tau) x for form 'Q'."""
        x = np.asarray(x).reshape(-1, self.nc)
        y = self.apply_D(x)
        if form == 'g5':
            return y - tau * self.g5c * x
        return self.g5c * y - tau * x

    def dense(self):
        n = int(np.prod(self.cdims)) * self.nc
        M = np.zeros((n, n), dtype=np.complex128)
        e = np.zeros(n, dtype=np.complex128)
        for j in range(n):
            e[j] = 1.0
            M[:, j] = self.apply_D(e).reshape(-1)
            e[j] = 0.0
        return M


# ----------------------------------------------------------------- fine operator forms
def fine_apply(op, psi, tau, form='g5'):
    """(D - tau Gamma5) psi (Eq. 3.7) or (Q - tau) psi (Eq. 3.6)."""
    if form == 'g5':
        return op.D_g5shift(psi, tau)
    return op.Q_shift(psi, tau)


# ----------------------------------------------------------------- SAP
class SAP:
    """Red-black multiplicative Schwarz smoother (Eq. 2.10, Proposition 1):
    one sweep applies, for colour 0 then colour 1, the block corrections
    x <- x + I_i A_i^{-1} I_i^H (b - A x) to all blocks i of that colour,
    with A_i = I_i^H A I_i the block restriction (hops leaving the block cut).
    Block solves are GMRES from zero to ``block_tol`` or ``block_iters``
    steps (Sec. 4, "Impact of the smoother"), or exact when ``exact`` is set.
    """

    def __init__(self, dims, block, block_iters=10, block_tol=1e-1, exact=False):
        self.blk = Blocking(dims, block)
        for e in self.blk.cdims:
            if e % 2:
                raise ValueError("SAP needs an even number of blocks in every direction")
        self.block_iters = block_iters
        self.block_tol = block_tol
        self.exact = exact
        self.members = [np.nonzero(self.blk.colour == c)[0] for c in range(2)]

    def _block_apply(self, apply_full, colour, vb):
        """A_i v_i for every block of one colour; vb (nbc, bs*12)."""
        blk = self.blk
        ids = self.members[colour]
        full = np.zeros((int(np.prod(blk.dims)), 4, 3), dtype=np.complex128)
        full[blk.sites[ids].reshape(-1)] = vb.reshape(-1, 4, 3)
        out = _flat(apply_full(full.reshape(blk.dims + (4, 3))))
        return out[blk.sites[ids]].reshape(len(ids), -1)

    def block_matrices(self, apply_full, colour):
        """Dense A_i for the blocks of one colour (exact-solve variant)."""
        n = self.blk.bsites * 12
        ids = self.members[colour]
        M = np.zeros((len(ids), n, n), dtype=np.complex128)
        for j in range(n):
            e = np.zeros((len(ids), n), dtype=np.complex128)
            e[:, j] = 1.0
            M[:, :, j] = self._block_apply(apply_full, colour, e)
        return M

    def sweep(self, apply_full, b, x):
        blk = self.blk
        for colour in (0, 1):
            r = _flat(b - apply_full(x))
            ids = self.members[colour]
            rb = r[blk.sites[ids]].reshape(len(ids), -1)
            if self.exact:
                M = self.block_matrices(apply_full, colour)
                eb = np.linalg.solve(M, rb[..., None])[..., 0]
            else:
                eb, _ = gmres(lambda v: self._block_apply(apply_full, colour, v), rb,
                              self.block_tol, self.block_iters)
            xf = _flat(x).copy()
            xf[blk.sites[ids].reshape(-1)] += eb.reshape(-1, 4, 3)
            x = xf.reshape(x.shape)
        return x

    def smooth(self, apply_full, b, x, sweeps):
        for _ in range(sweeps):
            x = self.sweep(apply_full, b, x)
        return x


# ----------------------------------------------------------------- two-level solver
class TwoLevelMG:
    """DD-alpha-AMG two-level preconditioner for (D - tau Gamma5) (Eq. 3.7) or
    (Q - tau) (Eq. 3.6): x = M b with
    x_c = GMRES(coarse operator, P^H b) to ``coarse_tol`` (Table 2: 5e-1),
    x = P x_c, then ``nu`` post-smoothing steps (Eq. 2.8 with mu = 0).

    ``smoother`` is 'sap' (SAP sweeps, Eq. 2.10) or 'gmres' (GMRES smoothing
    with ``smooth_iters`` steps, Sec. 2 last paragraph).
    """

    def __init__(self, op, agg_block, sap_block, nv, nu=4, coarse_tol=0.5,
                 coarse_maxiter=100, smoother='sap', sap_block_iters=10,
                 sap_block_tol=1e-1, smooth_iters=4, form='g5'):
        self.op = op
        self.agg_block = tuple(agg_block)
        self.nv = nv
        self.nu = nu
        self.coarse_tol = coarse_tol
        self.coarse_maxiter = coarse_maxiter
        self.smoother = smoother
        self.form = form
        self.smooth_iters = smooth_iters
        self.sap = SAP(op.dims, sap_block, sap_block_iters, sap_block_tol) if smoother == 'sap' else None
        self.interp = None
        self.coarse = None
        self.tau = 0.0

    def set_vectors(self, vectors):
        """Rebuild P and D_c from test vectors (Sec. 3, interpolation updates)."""
        self.interp = Interpolation(self.op.dims, self.agg_block, vectors)
        self.coarse = CoarseOperator.galerkin(self.op, self.interp)

    def fine(self, psi, tau=None):
        return fine_apply(self.op, psi, self.tau if tau is None else tau, self.form)

    def smooth(self, b, x, tau):
        A = lambda v: fine_apply(self.op, v, tau, self.form)
        if self.smoother == 'sap':
            return self.sap.smooth(A, b, x, self.nu)
        for _ in range(self.nu):
            r = (b - A(x)).reshape(1, -1)
            e, _ = gmres(lambda v: A(v.reshape(x.shape)).reshape(1, -1), r, 0.0, self.smooth_iters)
            x = x + e.reshape(x.shape)
        return x

    def coarse_solve(self, rc, tau):
        rc = rc.reshape(1, -1)
        xc, it = gmres(lambda v: self.coarse.apply(v, tau, self.form).reshape(1, -1), rc,
                       self.coarse_tol, self.coarse_maxiter)
        return xc.reshape(-1, self.interp.nc), int(it[0])

    def cycle(self, b, tau=None):
        tau = self.tau if tau is None else tau
        b = np.asarray(b).reshape(self.op.dims + (4, 3))
        rc = self.interp.restrict(b)
        xc, _ = self.coarse_solve(rc, tau)
        x = self.interp.prolong(xc)
        return self.smooth(b, x, tau)

    def solve(self, b, tau, tol=1e-1, maxiter=5, x0=None):
        """FGMRES preconditioned by the cycle (Sec. 4: stop at tol or maxiter)."""
        dims = self.op.dims
        A = lambda v: fine_apply(self.op, v.reshape(dims + (4, 3)), tau, self.form).reshape(-1)
        M = lambda v: self.cycle(v.reshape(dims + (4, 3)), tau).reshape(-1)
        x, it, res = fgmres(A, M, np.asarray(b).reshape(-1), tol, maxiter, x0)
        return x.reshape(dims + (4, 3)), it

    def setup(self, vectors, iterations=6):
        """Adaptive setup (Table 2: test vectors, setup iterations, smoothing
        steps); reading in the module header."""
        W = np.array(vectors, dtype=np.complex128).reshape((-1,) + self.op.dims + (4, 3))
        zero = np.zeros(self.op.dims + (4, 3), dtype=np.complex128)
        for i in range(W.shape[0]):
            W[i] = self.smooth(zero, W[i], 0.0)
            W[i] /= np.linalg.norm(W[i])
        self.set_vectors(W)
        for _ in range(iterations - 1):
            for i in range(W.shape[0]):
                W[i] = self.cycle(W[i], 0.0)
                W[i] /= np.linalg.norm(W[i])
            self.set_vectors(W)
        return W


# ----------------------------------------------------------------- three-level solver
class ThreeLevelMG(TwoLevelMG):
    """Three-level K-cycle (Sec. 2: the two-level construction applied
    recursively; Table 2's coarse tolerance at the middle level).  The fine
    level is ``TwoLevelMG``; its coarse solve becomes FGMRES on the level-1
    operator to ``coarse_tol`` (at most ``coarse_maxiter`` steps), right-
    preconditioned by the level-1 two-level cycle:
    x2 = GMRES(level-2 operator, P2^H r) to ``coarse2_tol``, x = P2 x2, then
    ``nu2`` GMRES smoothing steps of ``smooth2_iters`` iterations on the
    level-1 system.

    Readings taken where the paper is silent: the middle level smooths with
    GMRES (the paper's alternative smoother, Sec. 2 last paragraph) instead
    of SAP on the coarse lattice; without explicit level-2 test vectors, the
    first ``nv2`` fine test vectors restricted by P^H serve (they span the
    level-1 near-kernel that the fine test vectors carry down).
    """

    def __init__(self, op, agg_block, agg_block2, sap_block, nv, nv2, nu2=2, smooth2_iters=4,
                 coarse2_tol=0.5, coarse2_maxiter=100, **kw):
        super().__init__(op, agg_block, sap_block, nv, **kw)
        self.agg_block2 = tuple(agg_block2)
        self.nv2 = int(nv2)
        self.nu2 = int(nu2)
        self.smooth2_iters = int(smooth2_iters)
        self.coarse2_tol = coarse2_tol
        self.coarse2_maxiter = coarse2_maxiter
        self.interp2 = None
        self.coarse2 = None

    def set_vectors(self, vectors, vectors2=None):
        super().set_vectors(vectors)
        if vectors2 is None:
            W = np.asarray(vectors).reshape((-1,) + self.op.dims + (4, 3))
            if W.shape[0] < self.nv2:
                raise ValueError("need at least nv2 fine test vectors")
            vectors2 = [self.interp.restrict(W[i]).reshape(-1) for i in range(self.nv2)]
        self.interp2 = CoarseInterpolation(self.coarse.cdims, self.agg_block2, self.nv, vectors2)
        self.coarse2 = CoarseOperator.galerkin_coarse(self.coarse, self.interp2)

    def coarse_cycle(self, rc, tau):
        """The level-1 two-level cycle applied to a level-1 vector."""
        rc = np.asarray(rc).reshape(1, -1)
        A2 = lambda v: self.coarse2.apply(v, tau, self.form).reshape(1, -1)
        x2, _ = gmres(A2, self.interp2.restrict(rc).reshape(1, -1), self.coarse2_tol, self.coarse2_maxiter)
        x = self.interp2.prolong(x2).reshape(1, -1)
        A1 = lambda v: self.coarse.apply(v, tau, self.form).reshape(1, -1)
        for _ in range(self.nu2):
            e, _ = gmres(A1, rc - A1(x), 0.0, self.smooth2_iters)
            x = x + e
        return x.reshape(-1)

    def coarse_solve(self, rc, tau):
        A1 = lambda v: self.coarse.apply(v, tau, self.form).reshape(-1)
        M1 = lambda v: self.coarse_cycle(v, tau)
        xc, it, _ = fgmres(A1, M1, np.asarray(rc).reshape(-1), self.coarse_tol, self.coarse_maxiter)
        return xc.reshape(-1, self.interp.nc), int(it)
