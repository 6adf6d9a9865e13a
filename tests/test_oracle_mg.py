"""Pins of the oracle's multigrid pieces (no GPU): exact identities of Sec. 2
and Sec. 3 checked with dense matrices on small lattices, and brute-force
definitions of GMRES and SAP."""
import numpy as np
import pytest

from oracle.dirac import GAMMA5, WilsonClover
from oracle import mg
from paper_2004_08146_gb300 import synth


@pytest.fixture(scope="module")
def setting():
    dims = (4, 4, 4, 4)
    op = WilsonClover(synth.gauge_field(dims, 0.4, 77), -0.3, 1.2)
    vecs = synth.spinor(dims, 78, nvec=6)
    interp = mg.Interpolation(dims, (2, 2, 2, 2), vecs)
    P = interp.dense()
    coarse = mg.CoarseOperator.galerkin(op, interp)
    D = op.dense('D')
    return dict(dims=dims, op=op, vecs=vecs, interp=interp, P=P, coarse=coarse, D=D)


def _G5(V):
    return np.kron(np.eye(V), np.kron(GAMMA5, np.eye(3)))


def test_P_orthonormal_and_spin_structure(setting):
    """P^H P = I, and Gamma5 P = P Gamma5^c (Sec. 2, above Eq. 2.9)."""
    P = setting['P']
    interp = setting['interp']
    assert np.max(np.abs(P.conj().T @ P - np.eye(P.shape[1]))) < 1e-13
    V = int(np.prod(setting['dims']))
    g5c = np.tile(mg.gamma5_coarse(interp.nv), interp.blk.nblocks)
    assert np.max(np.abs(_G5(V) @ P - P * g5c[None, :])) < 1e-14


def test_range_contains_test_vectors(setting):
    """range(P) contains the test vectors it is built from (Sec. 3, "Local
    coherence"): P P^H w = w."""
    P = setting['P']
    for w in setting['vecs']:
        w = w.reshape(-1)
        assert np.linalg.norm(P @ (P.conj().T @ w) - w) < 1e-12 * np.linalg.norm(w)


@pytest.mark.slow
def test_rank_768_and_random_coherence():
    """24 test vectors, 2^4 aggregates on 4^4: dim range(P) = 24*2*16 = 768
    (Sec. 3 footnote), and for Gaussian random vectors E ||Pi v||^2/||v||^2 =
    768/3072 = 0.25 (the footnote's "no local coherence" value, read as the
    mean of lc^2)."""
    dims = (4, 4, 4, 4)
    interp = mg.Interpolation(dims, (2, 2, 2, 2), synth.spinor(dims, 5, nvec=24))
    P = interp.dense()
    assert P.shape[1] == 768
    assert np.linalg.matrix_rank(P) == 768
    R = synth.complex_gaussian((400, 3072), 6)
    proj = np.linalg.norm((R @ P.conj()) , axis=1) ** 2 / np.linalg.norm(R, axis=1) ** 2
    assert abs(proj.mean() - 0.25) < 0.01


def test_coarse_stencil_equals_dense_galerkin(setting):
    """The stencil D_c equals the dense P^H D P to 1e-13 (Eq. 2.8)."""
    P, D, coarse = setting['P'], setting['D'], setting['coarse']
    Dc = P.conj().T @ D @ P
    assert np.max(np.abs(coarse.dense() - Dc)) < 1e-13 * np.max(np.abs(Dc))


@pytest.mark.parametrize("dims,block", [((2, 2, 2, 2), (2, 2, 2, 2)),
                                        ((4, 2, 4, 2), (2, 2, 2, 2)),
                                        ((6, 2, 2, 4), (2, 2, 2, 2)),
                                        ((4, 4, 2, 2), (4, 2, 2, 2))])
def test_coarse_stencil_edge_extents(dims, block):
    """Coarse extents 1, 2 and 3 (hops that wrap into the same block, two
    directions landing on one neighbour block, odd coarse extent)."""
    op = WilsonClover(synth.gauge_field(dims, 0.5, 3), 0.2, 1.1)
    interp = mg.Interpolation(dims, block, synth.spinor(dims, 4, nvec=3))
    P = interp.dense()
    Dc = P.conj().T @ op.dense('D') @ P
    coarse = mg.CoarseOperator.galerkin(op, interp)
    assert np.max(np.abs(coarse.dense() - Dc)) < 1e-13 * np.max(np.abs(Dc))


def test_shift_rule_and_coarse_hermiticity(setting):
    """P^H (D - tau Gamma5) P = D_c - tau Gamma5^c and Q_c = Gamma5^c D_c is
    Hermitian (Sec. 2, Eq. 2.9)."""
    P, D, coarse = setting['P'], setting['D'], setting['coarse']
    V = int(np.prod(setting['dims']))
    tau = 0.37
    lhs = P.conj().T @ (D - tau * _G5(V)) @ P
    n = coarse.dense().shape[0]
    g5c = np.tile(coarse.g5c, n // coarse.nc)
    rhs = coarse.dense() - tau * np.diag(g5c)
    assert np.max(np.abs(lhs - rhs)) < 1e-13
    Qc = g5c[:, None] * coarse.dense()
    assert np.max(np.abs(Qc - Qc.conj().T)) < 1e-13
    x = synth.complex_gaussian((n,), 9)
    assert np.max(np.abs(coarse.apply(x, tau, 'g5').reshape(-1) - rhs @ x)) < 1e-12
    assert np.max(np.abs(coarse.apply(x, tau, 'Q').reshape(-1) - (Qc - tau * np.eye(n)) @ x)) < 1e-12


def test_coarse_grid_identity_eq_2_9(setting):
    """I - P Q_c^{-1} P^H Q = I - P D_c^{-1} P^H D (Eq. 2.9), dense."""
    P, D = setting['P'], setting['D']
    V = int(np.prod(setting['dims']))
    G5 = _G5(V)
    Q = G5 @ D
    Dc = P.conj().T @ D @ P
    Qc = P.conj().T @ Q @ P
    lhs = P @ np.linalg.solve(Qc, P.conj().T @ Q)
    rhs = P @ np.linalg.solve(Dc, P.conj().T @ D)
    assert np.max(np.abs(lhs - rhs)) < 1e-11


def test_restrict_prolong_are_P_adjoint_pair(setting):
    interp, P = setting['interp'], setting['P']
    r = synth.spinor(setting['dims'], 12)
    assert np.max(np.abs(interp.restrict(r).reshape(-1) - P.conj().T @ r.reshape(-1))) < 1e-13
    xc = synth.complex_gaussian((P.shape[1],), 13)
    assert np.max(np.abs(interp.prolong(xc).reshape(-1) - P @ xc)) < 1e-13


# ------------------------------------------------------------ GMRES
def test_gmres_equals_krylov_least_squares():
    """After k steps with tol 0, GMRES returns argmin_{x in K_k(A, b)} ||b - A x||
    (brute force: explicit Krylov basis and a least-squares solve)."""
    rng = np.random.default_rng(0)
    n = 40
    A = np.eye(n) * 3 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = synth.complex_gaussian((n,), 1)
    for k in (1, 3, 6):
        K = np.stack([np.linalg.matrix_power(A, j) @ b for j in range(k)], axis=1)
        y, *_ = np.linalg.lstsq(A @ K, b, rcond=None)
        xref = K @ y
        x, it = mg.gmres(lambda v: v @ A.T, b[None], 0.0, k)
        assert it[0] == k
        assert np.linalg.norm(x[0] - xref) < 1e-10 * np.linalg.norm(xref)


def test_gmres_batched_stopping():
    """Independent systems stop independently at their own tolerance."""
    n = 30
    A = np.diag(np.linspace(1, 2, n)).astype(complex)
    b = np.stack([synth.complex_gaussian((n,), 2), np.zeros(n) + 1.0], axis=0)
    b[1] = 0
    b[1, 0] = 1.0       # an eigenvector: solved exactly in one step
    x, it = mg.gmres(lambda v: v @ A.T, b, 1e-10, 25)
    assert it[1] == 1
    assert np.linalg.norm(A @ x[0] - b[0]) <= 1e-9 * np.linalg.norm(b[0])


def test_fgmres_exact_preconditioner_one_step():
    n = 25
    rng = np.random.default_rng(3)
    A = np.eye(n) * 2 + 0.3 * rng.standard_normal((n, n))
    Ainv = np.linalg.inv(A)
    b = synth.complex_gaussian((n,), 4)
    x, it, _ = mg.fgmres(lambda v: A @ v, lambda v: Ainv @ v, b, 1e-12, 5)
    assert it == 1
    assert np.linalg.norm(A @ x - b) < 1e-12 * np.linalg.norm(b)


# ------------------------------------------------------------ SAP
@pytest.fixture(scope="module")
def sap_setting():
    dims = (4, 4, 4, 4)
    op = WilsonClover(synth.gauge_field(dims, 0.5, 21), -0.2, 1.0)
    return dims, op


def test_sap_exact_sweep_equals_dense_product(sap_setting):
    """One SAP sweep with exact block solves is the product of the block
    projections of Eq. 2.10, applied block by block (red first), written with
    dense matrices."""
    dims, op = sap_setting
    tau = 0.1
    sap = mg.SAP(dims, (2, 2, 2, 2), exact=True)
    A = op.dense('Dg5', tau)
    b = synth.spinor(dims, 22).reshape(-1)
    x0 = synth.spinor(dims, 23).reshape(-1)
    x = x0.copy()
    blk = sap.blk
    for colour in (0, 1):
        for i in np.nonzero(blk.colour == colour)[0]:
            idx = (blk.sites[i][:, None] * 12 + np.arange(12)[None, :]).reshape(-1)
            Ai = A[np.ix_(idx, idx)]
            r = b - A @ x
            x[idx] += np.linalg.solve(Ai, r[idx])
    got = sap.sweep(lambda v: op.D_g5shift(v, tau), b.reshape(dims + (4, 3)), x0.reshape(dims + (4, 3)))
    assert np.linalg.norm(got.reshape(-1) - x) < 1e-12 * np.linalg.norm(x)


def test_sap_proposition_1(sap_setting):
    """Proposition 1 (Eq. 2.11): with exact block solves, SAP for (Q - tau) x = b
    and SAP for (D - tau Gamma5) x = Gamma5 b produce the same iterates."""
    dims, op = sap_setting
    tau = 0.23
    sap = mg.SAP(dims, (2, 2, 2, 2), exact=True)
    b = synth.spinor(dims, 24)
    x0 = synth.spinor(dims, 25)
    xq = sap.smooth(lambda v: op.Q_shift(v, tau), b, x0, 2)
    xd = sap.smooth(lambda v: op.D_g5shift(v, tau), op.g5(b), x0, 2)
    assert np.linalg.norm(xq - xd) < 1e-12 * np.linalg.norm(xd)


def test_sap_within_colour_order_independence(sap_setting):
    """Blocks of one colour are independent (Sec. 2, below Eq. 2.10): applying
    the GMRES block corrections of one colour one block at a time, in a
    permuted order and with the residual refreshed in between, gives the
    simultaneous result."""
    dims, op = sap_setting
    tau = -0.15
    A = lambda v: op.D_g5shift(v, tau)
    sap = mg.SAP(dims, (2, 2, 2, 2), block_iters=4, block_tol=0.0)
    b = synth.spinor(dims, 26)
    x0 = synth.spinor(dims, 27)
    simult = sap.sweep(A, b, x0)
    blk = sap.blk
    x = x0.reshape(-1, 4, 3).copy()
    rng = np.random.default_rng(5)
    for colour in (0, 1):
        ids = np.nonzero(blk.colour == colour)[0]
        for i in rng.permutation(ids):
            r = (b - A(x.reshape(x0.shape))).reshape(-1, 4, 3)
            mask = np.zeros(int(np.prod(dims)), bool)
            mask[blk.sites[i]] = True

            def Ai(v):
                full = np.zeros((int(np.prod(dims)), 4, 3), complex)
                full[blk.sites[i]] = v.reshape(-1, 4, 3)
                return A(full.reshape(x0.shape)).reshape(-1, 4, 3)[blk.sites[i]].reshape(1, -1)
            e, _ = mg.gmres(Ai, r[blk.sites[i]].reshape(1, -1), 0.0, 4)
            x[blk.sites[i]] += e.reshape(-1, 4, 3)
    assert np.linalg.norm(simult.reshape(-1) - x.reshape(-1)) < 1e-12 * np.linalg.norm(x)


def test_two_level_cycle_exact_coarse(setting):
    """Cycle with a (near) exact coarse solve and nu = 0 is P D_c^{-1} P^H b."""
    op, P, D = setting['op'], setting['P'], setting['D']
    dims = setting['dims']
    h = mg.TwoLevelMG(op, (2, 2, 2, 2), (2, 2, 2, 2), 6, nu=0, coarse_tol=1e-14,
                      coarse_maxiter=400, smoother='gmres')
    h.set_vectors(setting['vecs'])
    b = synth.spinor(dims, 30)
    got = h.cycle(b, 0.0).reshape(-1)
    Dc = P.conj().T @ D @ P
    ref = P @ np.linalg.solve(Dc, P.conj().T @ b.reshape(-1))
    assert np.linalg.norm(got - ref) < 1e-10 * np.linalg.norm(ref)


def test_local_coherence_measure():
    """lc(v) = ||Pi v|| / ||v|| (Sec. 3): 1 on the test vectors and on the range
    of P, P^H P = I (so Pi is an orthogonal projection), and for random
    vectors lc^2 averages to rank(P) / N = 768 / 3072 (the no-coherence value
    the paper quotes for this 4^4 setting with 24 vectors and 2^4 aggregates)."""
    dims = (4, 4, 4, 4)
    vecs = synth.spinor(dims, 71, nvec=24)
    interp = mg.Interpolation(dims, (2, 2, 2, 2), vecs)
    Pd = interp.dense()
    assert Pd.shape == (3072, 768)
    assert np.max(np.abs(Pd.conj().T @ Pd - np.eye(768))) < 1e-12
    for j in range(0, 24, 5):
        assert abs(mg.local_coherence(interp, vecs[j]) - 1.0) < 1e-12
    xc = synth.complex_gaussian((16, 2, 24), 72)
    assert abs(mg.local_coherence(interp, interp.prolong(xc)) - 1.0) < 1e-12
    rnd = synth.spinor(dims, 73, nvec=32)
    lc2 = np.array([mg.local_coherence(interp, rnd[j]) ** 2 for j in range(32)])
    assert abs(lc2.mean() - 0.25) < 0.02


def test_setup_enriches_the_near_kernel():
    """The adaptive setup has no unique result (only the solver's speed depends
    on it); what it must do is approximate the near-kernel of D.  On the 4^4
    field (smallest singular value of D = smallest |lambda(Q)| = 0.603) three
    setup iterations take ||D w|| / ||w|| of 8 random vectors from ~4.3 to
    below twice that singular value, and the vectors stay normalised."""
    from oracle.dirac import WilsonClover
    from oracle import mg
    dims = (4, 4, 4, 4)
    op = WilsonClover(synth.gauge_field(dims, 0.3, 1001), -0.2, 1.0)
    sigma_min = np.min(np.abs(np.linalg.eigvalsh(op.dense('Q'))))
    W0 = synth.spinor(dims, 5, nvec=8)
    before = np.array([np.linalg.norm(op.D(w)) / np.linalg.norm(w) for w in W0])
    W = mg.TwoLevelMG(op, (2, 2, 2, 2), (2, 2, 2, 2), 8).setup(W0.copy(), iterations=3)
    after = np.array([np.linalg.norm(op.D(w)) for w in W])
    assert np.allclose([np.linalg.norm(w) for w in W], 1.0, atol=1e-12)
    assert np.all(after >= sigma_min * (1 - 1e-12))
    assert np.all(after < 2.0 * sigma_min) and np.mean(after) < 0.25 * np.mean(before)


# ----------------------------------------------------------------- three levels
@pytest.fixture(scope="module")
def level1():
    dims = (8, 4, 4, 4)
    op = WilsonClover(synth.gauge_field(dims, 0.4, 31), -0.3, 1.2)
    vec = synth.spinor(dims, 32, nvec=4)
    I1 = mg.Interpolation(dims, (2, 2, 2, 2), vec)
    return op, vec, mg.CoarseOperator.galerkin(op, I1)


@pytest.mark.parametrize("block2", [(2, 1, 1, 1), (2, 2, 2, 2), (1, 2, 1, 2)])
def test_level2_interpolation_and_galerkin(level1, block2):
    """One level down (level-1 lattice 4 x 2^3, 2 N_v1 = 8): P2^H P2 = I,
    Gamma5^c P2 = P2 Gamma5^cc, P2 P2^H w = w for the level-2 test vectors,
    and the level-2 stencil equals dense P2^H D_c P2 (aggregate extents 1
    and 2, level-2 extents 1, 2 and 4)."""
    _, _, C1 = level1
    V1 = int(np.prod(C1.cdims))
    w2 = synth.complex_gaussian((3, V1 * C1.nc), 33)
    I2 = mg.CoarseInterpolation(C1.cdims, block2, C1.nv, w2)
    C2 = mg.CoarseOperator.galerkin_coarse(C1, I2)
    P2, D1, D2 = I2.dense(), C1.dense(), C2.dense()
    assert np.max(np.abs(P2.conj().T @ P2 - np.eye(P2.shape[1]))) < 1e-13
    g1 = np.tile(mg.gamma5_coarse(C1.nv), V1)
    g2 = np.tile(mg.gamma5_coarse(I2.nv), int(np.prod(C2.cdims)))
    assert np.max(np.abs(g1[:, None] * P2 - P2 * g2[None, :])) == 0.0
    for w in w2:
        assert np.linalg.norm(P2 @ (P2.conj().T @ w) - w) < 1e-12 * np.linalg.norm(w)
    assert np.max(np.abs(P2.conj().T @ D1 @ P2 - D2)) < 1e-13 * np.max(np.abs(D2))


def test_level1_cycle_is_coarse_grid_correction(level1):
    """Without middle-level smoothing and with an exact level-2 solve, the
    level-1 cycle is the coarse-grid correction P2 (P2^H A1 P2)^-1 P2^H r
    (Eq. 2.8 one level down), A1 = D_c - tau Gamma5^c."""
    op, vec, _ = level1
    h = mg.ThreeLevelMG(op, (2, 2, 2, 2), (2, 1, 1, 1), (2, 2, 2, 2), 4, 3, nu2=0,
                        coarse2_tol=1e-14, coarse2_maxiter=400)
    h.set_vectors(vec)
    tau = 0.07
    V1 = int(np.prod(h.coarse.cdims))
    A1 = h.coarse.dense() - tau * np.diag(np.tile(mg.gamma5_coarse(h.nv), V1))
    P2 = h.interp2.dense()
    r = synth.complex_gaussian((V1 * h.coarse.nc,), 35)
    ref = P2 @ np.linalg.solve(P2.conj().T @ A1 @ P2, P2.conj().T @ r)
    got = h.coarse_cycle(r, tau)
    assert np.linalg.norm(got - ref) < 1e-11 * np.linalg.norm(ref)


def test_k_cycle_with_exact_coarse_solve_is_two_level(level1):
    """Solving the level-1 system to 1e-13 inside the K-cycle gives the
    two-level cycle with an exact coarse solve, whatever the middle level
    does."""
    op, vec, _ = level1
    b = synth.spinor(op.dims, 34)
    two = mg.TwoLevelMG(op, (2, 2, 2, 2), (2, 2, 2, 2), 4, coarse_tol=1e-13, coarse_maxiter=400)
    two.set_vectors(vec)
    three = mg.ThreeLevelMG(op, (2, 2, 2, 2), (2, 1, 1, 1), (2, 2, 2, 2), 4, 3, coarse_tol=1e-13,
                            coarse_maxiter=400)
    three.set_vectors(vec)
    for tau in (0.0, 0.1):
        x2, x3 = two.cycle(b, tau), three.cycle(b, tau)
        assert np.linalg.norm(x3 - x2) < 1e-11 * np.linalg.norm(x2)


def test_three_level_solve_matches_dense():
    """FGMRES with the three-level K-cycle (Table 2 tolerances inside) solves
    (D - tau Gamma5) x = b on the 4^4 field to the dense solution."""
    dims = (4, 4, 4, 4)
    op = WilsonClover(synth.gauge_field(dims, 0.3, 1001), -0.2, 1.0)
    h = mg.ThreeLevelMG(op, (2, 2, 2, 2), (2, 2, 2, 2), (2, 2, 2, 2), 8, 6)
    h.set_vectors(synth.spinor(dims, 5, nvec=8))
    b = synth.spinor(dims, 6)
    x, it = h.solve(b, 0.05, tol=1e-12, maxiter=200)
    xd = np.linalg.solve(op.dense('Dg5', 0.05), b.reshape(-1))
    assert np.linalg.norm(x.reshape(-1) - xd) < 1e-10 * np.linalg.norm(xd)


@pytest.mark.parametrize("dims,block", [((4, 4, 4, 4), (2, 2, 2, 2)), ((8, 4, 2, 6), (4, 1, 2, 3)),
                                        ((6, 4, 4, 2), (3, 4, 1, 2))])
def test_blocking_gather_scatter_is_the_site_map(dims, block):
    """Blocking.gather / scatter (reshape form used by the restriction and
    prolongation) equal the explicit site map sites[b, l]."""
    blk = mg.Blocking(dims, block)
    f = synth.spinor(dims, 7)
    assert np.array_equal(blk.gather(f, (4, 3)), f.reshape(-1, 4, 3)[blk.sites])
    fb = synth.complex_gaussian((blk.nblocks, blk.bsites, 4, 3), 8)
    out = np.zeros((int(np.prod(dims)), 4, 3), dtype=np.complex128)
    out[blk.sites.reshape(-1)] = fb.reshape(-1, 4, 3)
    assert np.array_equal(blk.scatter(fb, (4, 3)), out.reshape(dims + (4, 3)))
