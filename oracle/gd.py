"""Generalized Davidson with harmonic Ritz extraction: GD-lambda-AMG in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Restates Algorithm 2 of the paper (Sec. 3): the search space V is extended by
the (approximate) solution t of the Gamma5-preconditioned correction equation
(D - theta Gamma5) t = Gamma5 r (Eq. 3.7); harmonic Ritz pairs come from the
pencil (QV)^H (QV) s = theta (QV)^H V s (Theorem 1, Eq. 3.5); converged pairs
are locked; at m_max the space is thick-restarted with the m_min harmonic
Ritz vectors of smallest |theta|; once n_tv eigenvectors are known the
interpolation is rebuilt from the n_tv locked vectors whose eigenvalues are
closest to the current target.

Readings taken where the paper leaves room:

* The pencil is solved as the Hermitian-definite problem
  (W^H V) s = mu (W^H W) s, mu = 1/theta (W = QV; W^H V = V^H Q V is
  Hermitian, W^H W positive definite): Cholesky of W^H W, then a Hermitian
  eigendecomposition.  Smallest |theta| = largest |mu|.
* Residual and reported eigenvalue use the Rayleigh quotient
  rho = u^H Q u of the normalised harmonic Ritz vector u (||r|| with rho is
  never larger than with theta).  The correction equation is shifted by rho
  as well (``shift='rho'``, default): while the residual is large the
  harmonic Ritz value can lie far outside the low spectrum (theta = -2.8
  against rho = -0.31 on the 16 x 8^3 workload), where SAP smoothing of
  D - theta Gamma5 stalls the iteration; both shifts agree at convergence.
  ``shift='theta'`` follows Algorithm 2 literally.
* Convergence: ||Q u - rho u||_2 <= eps_outer with ||u||_2 = 1.
* Locking removes the converged direction from the search space
  (V <- V C, W <- W C with C an orthonormal basis of s-perp), so V stays
  orthogonal to the locked vectors X without further operator applications;
  several pairs may lock in one iteration.
* Restart re-orthonormalises the retained harmonic Ritz vectors: with
  S = [s_1 .. s_mmin] and S = Q_S R_S, V <- V Q_S and W <- W Q_S.
* Orthogonalisation of t is classical Gram-Schmidt against V and then X,
  done twice.
* Output order: ascending |lambda|, ties by ascending lambda.
* Completion: once n pairs are locked, only harmonic Ritz values with |theta|
  below the n-th smallest locked |lambda| remain targets, and the run ends
  when none is left; the n locked pairs of smallest |lambda| are returned
  (the expansion follows a few targets at a time, so an eigenvalue can be
  locked after a larger one).  ``n_guard`` raises n by extra pairs.
"""
import numpy as np


def harmonic_ritz(V, W):
    """All harmonic Ritz pairs of Q w.r.t. span(V) given W = Q V (Theorem 1).

    Returns ``(theta, S)`` sorted by ascending |theta| (ties: ascending theta);
    columns of S are the coefficient vectors s (V s is the harmonic Ritz vector).
    """
    G = W.conj().T @ W
    Hm = W.conj().T @ V
    Hm = 0.5 * (Hm + Hm.conj().T)
    G = 0.5 * (G + G.conj().T)
    L = np.linalg.cholesky(G)
    Li = np.linalg.inv(L)
    C = Li @ Hm @ Li.conj().T
    C = 0.5 * (C + C.conj().T)
    mu, Y = np.linalg.eigh(C)
    S = Li.conj().T @ Y
    with np.errstate(divide='ignore'):
        theta = np.where(mu != 0, 1.0 / np.where(mu != 0, mu, 1.0), np.inf)
    order = np.lexsort((theta, np.abs(theta)))
    return theta[order], S[:, order]


def rayleigh_ritz(V, W):
    """All Ritz pairs of Q w.r.t. span(V) for orthonormal V, given W = Q V:
    the Ritz-Galerkin condition Q u - theta u orthogonal to span(V) (Sec. 3)
    reduces to the Hermitian eigenproblem (V^H Q V) s = theta s.

    Returns ``(theta, S)`` in the order of ``harmonic_ritz``.
    """
    Hm = V.conj().T @ W
    Hm = 0.5 * (Hm + Hm.conj().T)
    theta, S = np.linalg.eigh(Hm)
    order = np.lexsort((theta, np.abs(theta)))
    return theta[order], S[:, order]


def _orth_complement(s):
    """Orthonormal basis of the complement of unit vector s in C^m."""
    m = s.shape[0]
    Qf, _ = np.linalg.qr(np.concatenate([s[:, None], np.eye(m, dtype=np.complex128)], axis=1))
    return Qf[:, 1:m]


class GDResult:
    def __init__(self, lam, X, outer, inner, converged, residuals):
        self.lam = lam
        self.X = X
        self.outer = outer
        self.inner = inner
        self.converged = converged
        self.residuals = residuals


def select_targets(theta, b, candidates=None):
    """Indices of the b targets among harmonic Ritz values sorted by |theta|.

    b = 1 is Algorithm 2's rule (smallest |theta|).  For b > 1 the targets
    alternate between the two signs, starting with the sign of the smallest
    |theta| and taking each sign's values by ascending |theta| (reading: the
    block variant keeps both halves of the indefinite spectrum in the search
    space).  ``candidates`` restricts the choice to a subset of indices.
    """
    order = np.arange(theta.size) if candidates is None else np.asarray(candidates, dtype=np.int64)
    if order.size == 0:
        return order
    if b <= 1 or order.size <= 1:
        return order[:1]
    first = theta[order[0]] >= 0
    same = [i for i in order if (theta[i] >= 0) == first]
    other = [i for i in order if (theta[i] >= 0) != first]
    out = []
    while len(out) < min(b, order.size):
        if same:
            out.append(same.pop(0))
        if len(out) < b and other:
            out.append(other.pop(0))
    return np.asarray(out[:b])


def gd_lambda_amg(Q, n, V0, t0, correction, m_min=30, m_max=50, eps=1e-8,
                  n_tv=None, on_update=None, update_every=1, max_outer=100000,
                  random_vector=None, n_guard=0, block=1, shift='rho', extraction='harmonic',
                  confirm=0):
    """Algorithm 2 (GD-lambda-AMG) on flat complex vectors.

    Q            : callable, v (N,) -> Q v
    n            : number of eigenpairs sought
    V0           : (N, n_tv) initial guess columns (e.g. setup test vectors)
    t0           : (N,) or (N, block) initial expansion vector(s)
    correction   : callable (theta, r) -> (t, inner_iterations); approximate
                   solution of the correction equation (Eq. 3.6 / Eq. 3.7)
    on_update    : callable (vectors (N, n_tv)) rebuilding the interpolation;
                   called after a lock once len(X) >= n_tv, every
                   ``update_every`` locks
    n_guard      : extra pairs to lock before stopping; the n smallest |lambda|
                   of the n + n_guard locked pairs are returned (an interior
                   eigensolver can skip an eigenvalue near the end of its run)
    block        : number of targets (and correction solves) per outer
                   iteration, chosen by ``select_targets``; 1 = Algorithm 2
    shift        : 'rho' shifts the correction equation by the Rayleigh
                   quotient of the target vector, 'theta' by its harmonic
                   Ritz value (Algorithm 2 as printed)
    extraction   : 'harmonic' (Theorem 1, the method's default) or 'rr' for
                   the Rayleigh-Ritz pairs (the comparison of Sec. 4)
    confirm      : completion check (the paper states no stopping rule beyond
                   the number of pairs): once n pairs are locked and no
                   harmonic Ritz value lies below the n-th smallest locked
                   |lambda|, the run continues until this many correction
                   equations (for the smallest values above that bound) have
                   left none below it; a value below it resets the count
    """
    extract = harmonic_ritz if extraction == 'harmonic' else rayleigh_ritz
    n_want = n
    n = n + int(n_guard)
    V0 = np.asarray(V0, dtype=np.complex128)
    N = V0.shape[0]
    n_tv = V0.shape[1] if n_tv is None else n_tv
    X = np.zeros((N, 0), dtype=np.complex128)
    lam = []
    res = []
    V, _ = np.linalg.qr(V0)
    W = np.stack([Q(V[:, j]) for j in range(V.shape[1])], axis=1)
    T = np.asarray(t0, dtype=np.complex128).reshape(N, -1).copy()
    rnd = random_vector if random_vector is not None else \
        (lambda k: np.random.default_rng(k).standard_normal(N) + 0j)
    outer = 0
    inner = 0
    locks_since_update = 0
    finished = False
    confirm_done = 0
    while not finished and outer < max_outer:
        outer += 1
        added = 0
        for j in range(T.shape[1]):
            t = T[:, j]
            for _ in range(2):
                t = t - V @ (V.conj().T @ t)
                if X.shape[1]:
                    t = t - X @ (X.conj().T @ t)
            nt = np.linalg.norm(t)
            if not np.isfinite(nt) or nt < 1e-12:
                continue
            v = t / nt
            V = np.concatenate([V, v[:, None]], axis=1)
            W = np.concatenate([W, Q(v)[:, None]], axis=1)
            added += 1
        if added == 0:
            T = rnd(outer)[:, None]
            continue
        finished = False
        confirming = False
        while True:
            theta, S = extract(V, W)
            cand = None
            if len(lam) >= n:
                lim = np.sort(np.abs(lam))[n - 1]
                cand = np.nonzero(np.abs(theta) < lim)[0]
                confirming = cand.size == 0
                if confirming:
                    if confirm_done >= confirm:
                        finished = True
                        break
                    cand = None
                else:
                    confirm_done = 0
            tg = select_targets(theta, block, cand)
            pairs = []
            locked = False
            for k in tg:
                s = S[:, k] / np.linalg.norm(V @ S[:, k])
                u = V @ s
                Qu = W @ s
                rho = float(np.real(np.vdot(u, Qu)))
                r = Qu - rho * u
                rn = np.linalg.norm(r)
                if rn <= eps:
                    lam.append(rho)
                    res.append(rn)
                    X = np.concatenate([X, u[:, None]], axis=1)
                    C = _orth_complement(s / np.linalg.norm(s))
                    V = V @ C
                    W = W @ C
                    locks_since_update += 1
                    locked = True
                    break
                pairs.append((rho if shift == 'rho' else float(theta[k]), r))
            if not locked:
                break
            if V.shape[1] == 0:
                break
            if on_update is not None and X.shape[1] >= n_tv and locks_since_update >= update_every:
                theta2, _ = extract(V, W)
                target = theta2[0]
                dist = np.abs(np.asarray(lam) - target)
                pick = np.lexsort((np.arange(len(lam)), dist))[:n_tv]
                on_update(X[:, np.sort(pick)])
                locks_since_update = 0
        if finished:
            break
        if V.shape[1] == 0:
            T = rnd(outer)[:, None]
            continue
        T = np.zeros((N, len(pairs)), dtype=np.complex128)
        for j, (th, r) in enumerate(pairs):
            t, it = correction(th, r)
            T[:, j] = t
            inner += int(it)
        if confirming:
            confirm_done += len(pairs)
        if V.shape[1] + T.shape[1] > m_max:
            theta, S = extract(V, W)
            Qs, _ = np.linalg.qr(S[:, :m_min])
            V = V @ Qs
            W = W @ Qs
    lam = np.asarray(lam)
    order = np.lexsort((lam, np.abs(lam)))[:n_want]
    return GDResult(lam[order], X[:, order], outer, inner, finished, np.asarray(res)[order])
