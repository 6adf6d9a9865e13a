"""Pins of the oracle's generalized Davidson (no GPU): Theorem 1, the
Gamma5-preconditioning equivalence and a brute-force dense eigendecomposition
at 4^4 (the small lattice the paper itself diagonalises fully, Sec. 3)."""
import numpy as np
import pytest

from oracle.dirac import WilsonClover
from oracle import gd, mg
from paper_2004_08146_gb300 import synth


def _herm(n, seed):
    A = synth.complex_gaussian((n, n), seed)
    return 0.5 * (A + A.conj().T)


def test_theorem_1_harmonic_pencil():
    """Theorem 1: the pencil W^H A V s = theta W^H V s (W = A V) has the
    eigenvalues of H_m = (W^H V)^{-1} W^H A V."""
    n, m = 60, 8
    A = _herm(n, 1)
    V, _ = np.linalg.qr(synth.complex_gaussian((n, m), 2))
    W = A @ V
    theta, S = gd.harmonic_ritz(V, W)
    Hm = np.linalg.solve(W.conj().T @ V, W.conj().T @ A @ V)
    ev = np.linalg.eigvals(Hm)
    assert np.max(np.abs(np.sort_complex(ev) - np.sort_complex(theta.astype(complex)))) < 1e-9
    for k in range(m):   # (W^H W) s = theta (W^H V) s column by column
        s = S[:, k]
        assert np.linalg.norm(W.conj().T @ W @ s - theta[k] * (W.conj().T @ V @ s)) < 1e-9 * np.linalg.norm(W.conj().T @ W @ s)
    assert np.all(np.diff(np.abs(theta)) >= -1e-15)


def test_harmonic_ritz_invariant_subspace_exact():
    """If span(V) is invariant, the harmonic Ritz values are exact eigenvalues."""
    n = 50
    A = _herm(n, 3)
    lam, U = np.linalg.eigh(A)
    idx = [3, 10, 22, 40]
    V, _ = np.linalg.qr(U[:, idx] @ synth.complex_gaussian((4, 4), 4))
    theta, _ = gd.harmonic_ritz(V, A @ V)
    assert np.max(np.abs(np.sort(theta) - np.sort(lam[idx]))) < 1e-12


def test_gamma5_preconditioned_equivalence():
    """(Q - tau) t = r  <=>  (D - tau Gamma5) t = Gamma5 r (Eq. 3.6, Eq. 3.7)."""
    dims = (2, 2, 2, 4)
    op = WilsonClover(synth.gauge_field(dims, 0.5, 5), -0.1, 1.2)
    tau = 0.31
    r = synth.spinor(dims, 6).reshape(-1)
    t1 = np.linalg.solve(op.dense('Q', tau), r)
    t2 = np.linalg.solve(op.dense('Dg5', tau), op.g5(r.reshape(dims + (4, 3))).reshape(-1))
    assert np.linalg.norm(t1 - t2) < 1e-12 * np.linalg.norm(t1)


def test_select_targets():
    th = np.array([-0.1, -0.2, 0.25, -0.3, 0.4, 0.5])
    assert list(gd.select_targets(th, 1)) == [0]
    assert list(gd.select_targets(th, 2)) == [0, 2]
    assert list(gd.select_targets(th, 4)) == [0, 2, 1, 4]


@pytest.mark.slow
def test_gd_c1_matches_dense_eig():
    """GD with plain GMRES inner solves on the 4^4 workload (eps 0.3, csw 1.0,
    m0 = -0.2): the 10 smallest |lambda| of the 3072 x 3072 Q from dense eigh,
    relative error <= 1e-10 and residual <= 1e-8."""
    dims = (4, 4, 4, 4)
    op = WilsonClover(synth.gauge_field(dims, 0.3, 1001), -0.2, 1.0)
    M = op.dense('Q')
    ev = np.linalg.eigvalsh(M)
    ev = ev[np.lexsort((ev, np.abs(ev)))]
    N = op.n
    Q = lambda v: op.Q(v.reshape(dims + (4, 3))).reshape(-1)

    def corr(theta, r):
        x, it = mg.gmres(lambda v: (M @ v[0] - theta * v[0])[None], r[None], 1e-1, 20)
        return x[0], it[0]
    res = gd.gd_lambda_amg(Q, 10, synth.complex_gaussian((N, 8), 7), synth.complex_gaussian((N, 2), 8),
                           corr, m_min=30, m_max=50, eps=1e-8, block=2)
    assert res.converged
    assert np.max(np.abs(res.lam - ev[:10]) / np.abs(ev[:10])) < 1e-10
    for j in range(10):
        u = res.X[:, j]
        assert abs(np.linalg.norm(u) - 1) < 1e-12
        assert np.linalg.norm(Q(u) - res.lam[j] * u) <= 1e-8


def test_rayleigh_ritz_galerkin_condition():
    """Rayleigh-Ritz pairs (Sec. 3): A u - theta u is orthogonal to span(V)
    for u = V s, and an invariant subspace gives exact eigenpairs."""
    n, m = 60, 8
    A = _herm(n, 3)
    V, _ = np.linalg.qr(synth.complex_gaussian((n, m), 4))
    theta, S = gd.rayleigh_ritz(V, A @ V)
    assert np.all(np.diff(np.abs(theta)) >= 0)
    for k in range(m):
        u = V @ S[:, k]
        assert np.linalg.norm(V.conj().T @ (A @ u - theta[k] * u)) < 1e-12 * np.linalg.norm(A)
    w, Y = np.linalg.eigh(A)
    theta2, S2 = gd.rayleigh_ritz(Y[:, 10:18], A @ Y[:, 10:18])
    assert np.max(np.abs(np.sort(theta2) - np.sort(w[10:18]))) < 1e-12 * np.max(np.abs(w))



@pytest.mark.slow
def test_gd_three_level_corrections_c1():
    """GD-lambda-AMG whose correction equations (Eq. 3.7) are solved by FGMRES
    with the three-level K-cycle (4^4 -> 2^4 -> 1^4, Nv 8 then 6; Table 2
    tolerances): the 10 smallest |lambda| of the dense Q to 1e-10."""
    dims = (4, 4, 4, 4)
    op = WilsonClover(synth.gauge_field(dims, 0.3, 1001), -0.2, 1.0)
    ev = np.linalg.eigvalsh(op.dense('Q'))
    ev = ev[np.lexsort((ev, np.abs(ev)))]
    Q = lambda v: op.Q(v.reshape(dims + (4, 3))).reshape(-1)
    h = mg.ThreeLevelMG(op, (2, 2, 2, 2), (2, 2, 2, 2), (2, 2, 2, 2), 8, 6)
    W = h.setup(synth.spinor(dims, 11, nvec=8), iterations=3)

    def corr(theta, r):
        x, it = h.solve(op.g5(r.reshape(dims + (4, 3))), theta, 1e-1, 5)
        return x.reshape(-1), it
    res = gd.gd_lambda_amg(Q, 10, W.reshape(8, -1).T, synth.complex_gaussian((op.n, 2), 12), corr,
                           m_min=30, m_max=50, eps=1e-8, block=2)
    assert res.converged
    assert np.max(np.abs(res.lam - ev[:10]) / np.abs(ev[:10])) < 1e-10


def test_completion_confirm_passes():
    """The completion check: with confirm = 0 the run ends at the first check
    that finds no harmonic Ritz value below the k-th locked |lambda|; with
    confirm = 8 corrections (two outer iterations of 4 targets) the same
    (deterministic) run reaches that check at the same outer iteration and
    then takes at least two more.  Both return the k smallest |lambda| of a
    dense Hermitian indefinite matrix with a cluster at the k-th value."""
    n, k = 120, 10
    w = np.concatenate([np.linspace(0.05, 1.0, n // 2), -np.linspace(0.06, 1.1, n // 2)])
    w[:6] = 0.2 + 1e-3 * np.arange(6)          # a cluster around the boundary
    Y, _ = np.linalg.qr(synth.complex_gaussian((n, n), 6))
    A = (Y * w) @ Y.conj().T
    A = 0.5 * (A + A.conj().T)
    ev = w[np.lexsort((w, np.abs(w)))]

    def corr(theta, r):
        x, it = mg.gmres(lambda v: (A @ v[0] - theta * v[0])[None], r[None], 1e-1, 8)
        return x[0], it[0]
    out = {}
    for c in (0, 8):
        out[c] = gd.gd_lambda_amg(lambda v: A @ v, k, synth.complex_gaussian((n, 6), 7),
                                  synth.complex_gaussian((n, 4), 8), corr, m_min=16, m_max=32,
                                  eps=1e-9, block=4, confirm=c)
        assert out[c].converged
        assert np.max(np.abs(out[c].lam - ev[:k]) / np.abs(ev[:k])) < 1e-10
    assert out[8].outer >= out[0].outer + 2


def test_guard_pairs_return_the_k_smallest():
    """Guard pairs: the completion check runs on k + g locked pairs and the k
    smallest |lambda| are returned -- still exactly the k smallest of a dense
    Hermitian indefinite matrix, after at least as many outer iterations as
    without guard pairs (the same deterministic run up to the first check)."""
    n, k = 120, 10
    w = np.concatenate([np.linspace(0.05, 1.0, n // 2), -np.linspace(0.06, 1.1, n // 2)])
    w[:6] = 0.2 + 1e-3 * np.arange(6)
    Y, _ = np.linalg.qr(synth.complex_gaussian((n, n), 6))
    A = (Y * w) @ Y.conj().T
    A = 0.5 * (A + A.conj().T)
    ev = w[np.lexsort((w, np.abs(w)))]

    def corr(theta, r):
        x, it = mg.gmres(lambda v: (A @ v[0] - theta * v[0])[None], r[None], 1e-1, 8)
        return x[0], it[0]
    out = {}
    for g in (0, 4):
        out[g] = gd.gd_lambda_amg(lambda v: A @ v, k, synth.complex_gaussian((n, 6), 7),
                                  synth.complex_gaussian((n, 4), 8), corr, m_min=16, m_max=32,
                                  eps=1e-9, block=4, n_guard=g)
        assert out[g].converged and out[g].lam.size == k
        assert np.max(np.abs(out[g].lam - ev[:k]) / np.abs(ev[:k])) < 1e-10
    assert out[4].outer >= out[0].outer
