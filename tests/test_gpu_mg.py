"""GPU parity of the multigrid pieces against the FP64 oracle through the C
ABI: P (Sec. 2 above Eq. 2.9), P^H / P, the Galerkin stencil (Eq. 2.8, 2.9),
the coarse apply, SAP sweeps (Eq. 2.10), one two-level cycle and the shifted
solve.  Fixed iteration counts (tolerance 0) make the Krylov pieces
comparable step by step; FP64 agrees to rounding (1e-10 relative after the
GMRES steps), FP32 to 1e-4."""
import numpy as np
import pytest

from oracle.dirac import WilsonClover
from oracle import mg
from paper_2004_08146_gb300 import synth
from gpu_util import make_ctx, dev, host, relerr, torch_cuda

pytestmark = pytest.mark.gpu

DIMS = (8, 4, 4, 4)
BLOCK = (2, 2, 2, 2)
NV = 6


@pytest.fixture(scope="module")
def setting():
    torch_cuda()
    U = synth.gauge_field(DIMS, 0.5, 51)
    m0, csw = -0.3, 1.3
    op = WilsonClover(U, m0, csw)
    vecs = synth.spinor(DIMS, 52, nvec=NV)
    interp = mg.Interpolation(DIMS, BLOCK, vecs)
    coarse = mg.CoarseOperator.galerkin(op, interp)
    ctx = make_ctx(U, DIMS, m0, csw, sap_block=BLOCK, sap_block_iters=4, sap_block_tol=-1.0,
                   coarse_tol=0.0, coarse_maxiter=8, nu=2, precision=0)
    V = dev(vecs)
    ctx.qcd_mg_update_from_eigvecs(V, NV)
    return dict(U=U, op=op, vecs=vecs, interp=interp, coarse=coarse, ctx=ctx, m0=m0, csw=csw)


def test_P_matches_oracle(setting):
    P = setting["ctx"].qcd_mg_get_P()
    assert relerr(P, setting["interp"].P) < 1e-12


def test_coarse_stencil_matches_oracle(setting):
    A = setting["ctx"].qcd_mg_get_coarse()
    ref = setting["coarse"].A
    assert np.max(np.abs(A - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 2e-6)])
def test_restrict_prolong(setting, prec, tol):
    torch = torch_cuda()
    ctx, interp = setting["ctx"], setting["interp"]
    dt = np.complex128 if prec == 0 else np.complex64
    nrhs = 2
    r = synth.spinor(DIMS, 53, nvec=nrhs)
    info = ctx.qcd_mg_info()
    ncoarse = info["coarse_sites"] * 2 * NV
    xc = torch.zeros(nrhs * ncoarse, dtype=torch.complex128 if prec == 0 else torch.complex64, device="cuda")
    ctx.qcd_mg_restrict(prec, nrhs, dev(r, dt), xc)
    got = host(xc).reshape(nrhs, -1)
    for j in range(nrhs):
        assert relerr(got[j], interp.restrict(r[j]).reshape(-1)) < tol
    c = synth.complex_gaussian((nrhs, ncoarse), 54)
    x = dev(r, dt)
    ctx.qcd_mg_prolong(prec, nrhs, dev(c, dt), x)
    got = host(x).reshape(nrhs, -1)
    for j in range(nrhs):
        assert relerr(got[j], interp.prolong(c[j]).reshape(-1)) < tol


@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 2e-6)])
def test_coarse_apply_both_forms(setting, prec, tol):
    from paper_2004_08146_gb300 import qcd
    ctx, coarse = setting["ctx"], setting["coarse"]
    dt = np.complex128 if prec == 0 else np.complex64
    info = ctx.qcd_mg_info()
    n = info["coarse_sites"] * 2 * NV
    x = synth.complex_gaussian((2, n), 55)
    taus = [0.13, -0.4]
    for op, form in ((qcd.QCD_OP_D, 'g5'), (qcd.QCD_OP_Q, 'Q')):
        xd = dev(x, dt)
        y = xd.clone()
        ctx.qcd_coarse_apply(op, prec, 2, xd, y, taus)
        got = host(y).reshape(2, -1)
        for j in range(2):
            assert relerr(got[j], coarse.apply(x[j], taus[j], form).reshape(-1)) < tol


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
def test_sap_sweeps_fixed_iterations(setting, prec, tol):
    from paper_2004_08146_gb300 import qcd
    ctx, op = setting["ctx"], setting["op"]
    dt = np.complex128 if prec == 0 else np.complex64
    b = synth.spinor(DIMS, 56, nvec=2)
    x0 = synth.spinor(DIMS, 57, nvec=2)
    taus = [0.1, -0.2]
    for opc, form in ((qcd.QCD_OP_D, 'g5'), (qcd.QCD_OP_Q, 'Q')):
        xd = dev(x0, dt)
        ctx.qcd_sap(opc, prec, 2, dev(b, dt), xd, taus, 2, -1.0)
        got = host(xd).reshape((2,) + DIMS + (4, 3))
        sap = mg.SAP(DIMS, BLOCK, block_iters=4, block_tol=0.0)
        for j in range(2):
            A = lambda v, t=taus[j]: mg.fine_apply(op, v, t, form)
            ref = sap.smooth(A, b[j], x0[j], 2)
            assert relerr(got[j], ref) < tol


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
def test_two_level_cycle(setting, prec, tol):
    from paper_2004_08146_gb300 import qcd
    ctx, op = setting["ctx"], setting["op"]
    dt = np.complex128 if prec == 0 else np.complex64
    b = synth.spinor(DIMS, 58, nvec=1)
    tau = [0.07]
    h = mg.TwoLevelMG(op, BLOCK, BLOCK, NV, nu=2, coarse_tol=0.0, coarse_maxiter=8, smoother='sap',
                      sap_block_iters=4, sap_block_tol=0.0)
    h.set_vectors(setting["vecs"])
    ref = h.cycle(b[0], tau[0])
    x = dev(b, dt)
    ctx.qcd_mg_cycle(qcd.QCD_OP_D, prec, 1, dev(b, dt), x, tau)
    assert relerr(host(x), ref) < tol


@pytest.mark.parametrize("precision", [0, 1])
def test_shifted_solve_residual(setting, precision):
    """(Q - tau) x = b to 1e-10 relative (Eq. 1.1) with FP64 refinement; the
    residual is measured by the oracle operator."""
    from paper_2004_08146_gb300 import qcd
    torch = torch_cuda()
    U, op = setting["U"], setting["op"]
    ctx = make_ctx(U, DIMS, setting["m0"], setting["csw"], sap_block=BLOCK, precision=precision)
    ctx.qcd_mg_setup(NV, BLOCK)
    b = synth.spinor(DIMS, 59, nvec=3)
    taus = [0.0, 0.15, -0.3]
    bs = [dev(b[j]) for j in range(3)]
    xs = [torch.zeros_like(bs[0]) for _ in range(3)]
    rc, info = ctx.qcd_shifted_solve_batched(bs, xs, taus, 1e-10)
    assert rc == qcd.QCD_OK
    for j in range(3):
        xh = host(xs[j]).reshape(DIMS + (4, 3))
        res = np.linalg.norm(b[j] - op.Q_shift(xh, taus[j])) / np.linalg.norm(b[j])
        assert res < 2e-10


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
def test_two_level_cycle_gmres_smoother(setting, prec, tol):
    """The cycle with the GMRES smoother (Sec. 2, last paragraph) in both forms
    of the shifted operator, D - tau Gamma5 (Eq. 3.7) and Q - tau (Eq. 3.6)."""
    from paper_2004_08146_gb300 import qcd
    op = setting["op"]
    dt = np.complex128 if prec == 0 else np.complex64
    ctx = make_ctx(setting["U"], DIMS, setting["m0"], setting["csw"], sap_block=BLOCK, smoother=1,
                   gmres_smooth_iters=3, nu=2, coarse_tol=0.0, coarse_maxiter=8, precision=0)
    ctx.qcd_mg_update_from_eigvecs(dev(setting["vecs"]), NV)
    b = synth.spinor(DIMS, 61, nvec=1)
    tau = [0.11]
    for form, oform in ((qcd.QCD_OP_D, 'g5'), (qcd.QCD_OP_Q, 'Q')):
        h = mg.TwoLevelMG(op, BLOCK, BLOCK, NV, nu=2, coarse_tol=0.0, coarse_maxiter=8, smoother='gmres',
                          smooth_iters=3, form=oform)
        h.set_vectors(setting["vecs"])
        ref = h.cycle(b[0], tau[0])
        x = dev(b, dt)
        ctx.qcd_mg_cycle(form, prec, 1, dev(b, dt), x, tau)
        assert relerr(host(x), ref) < tol, form


def test_local_coherence_matches_oracle():
    """lc(v) = ||Pi v|| / ||v|| (Sec. 3) through the C ABI against the oracle's
    projection P (P^H v): eigenvectors of the 4^4 Q, with P built from the 24
    eigenvectors closest to zero (2^4 aggregates, as in the paper's 4^4 study)."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 1001)
    op = WilsonClover(U, -0.2, 1.0)
    w, Y = np.linalg.eigh(op.dense('Q'))
    near = np.argsort(np.abs(w))[:24]
    vecs = Y[:, near].T.reshape((24,) + dims + (4, 3))
    ctx = make_ctx(U, dims, -0.2, 1.0, sap_block=(2, 2, 2, 2), precision=0)
    ctx.qcd_mg_update_from_eigvecs(dev(vecs), 24)
    interp = mg.Interpolation(dims, (2, 2, 2, 2), vecs)
    pick = np.arange(0, 3072, 16)
    sample = Y[:, pick].T.copy()
    got = ctx.qcd_local_coherence(len(pick), dev(sample))
    ref = np.array([mg.local_coherence(interp, sample[j]) for j in range(len(pick))])
    assert np.max(np.abs(got - ref)) < 1e-12
    own = ctx.qcd_local_coherence(24, dev(vecs))
    assert np.max(np.abs(own - 1.0)) < 1e-12
