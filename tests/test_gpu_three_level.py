"""GPU parity of the three-level hierarchy against the oracle's
``ThreeLevelMG`` through the C ABI: P2 and the level-2 Galerkin stencil
(element by element), one K-cycle with fixed iteration counts (FP64 to
rounding, FP32 to 1e-4), and a shifted solve with the K-cycle inside."""
import numpy as np
import pytest

from oracle.dirac import WilsonClover
from oracle import mg
from paper_2004_08146_gb300 import synth
from gpu_util import make_ctx, dev, host, relerr, torch_cuda

pytestmark = pytest.mark.gpu

DIMS = (8, 4, 4, 4)
BLOCK = (2, 2, 2, 2)
AGG2 = (2, 1, 1, 1)
NV, NV2 = 6, 4
KC = dict(coarse_tol=0.0, coarse_maxiter=4, nu=2, sap_block_iters=4, gmres_smooth_iters=3, nu2=2)


@pytest.fixture(scope="module")
def setting():
    torch_cuda()
    U = synth.gauge_field(DIMS, 0.5, 51)
    m0, csw = -0.3, 1.3
    op = WilsonClover(U, m0, csw)
    vecs = synth.spinor(DIMS, 52, nvec=NV)
    h = mg.ThreeLevelMG(op, BLOCK, AGG2, BLOCK, NV, NV2, nu2=KC["nu2"], smooth2_iters=KC["gmres_smooth_iters"],
                        coarse2_tol=0.0, coarse2_maxiter=KC["coarse_maxiter"], nu=KC["nu"], coarse_tol=0.0,
                        coarse_maxiter=KC["coarse_maxiter"], smoother='sap', sap_block_iters=KC["sap_block_iters"],
                        sap_block_tol=0.0)
    h.set_vectors(vecs)
    ctx = make_ctx(U, DIMS, m0, csw, sap_block=BLOCK, sap_block_tol=-1.0, precision=0, levels=3, nv2=NV2,
                   agg2=AGG2, **KC)
    ctx.qcd_mg_update_from_eigvecs(dev(vecs), NV)
    return dict(U=U, op=op, vecs=vecs, h=h, ctx=ctx, m0=m0, csw=csw)


def test_level2_sizes(setting):
    info = setting["ctx"].qcd_mg_info2()
    assert info["dims"] == (2, 2, 2, 2) and info["nv2"] == NV2 and info["nv1"] == NV
    assert info["aggregate_sites"] == 2 and info["sites"] == 16


def test_P2_matches_oracle(setting):
    P2 = setting["ctx"].qcd_mg_get_P2()
    assert relerr(P2, setting["h"].interp2.P) < 1e-12


def test_level2_stencil_matches_oracle(setting):
    A2 = setting["ctx"].qcd_mg_get_coarse2()
    ref = setting["h"].coarse2.A
    assert np.max(np.abs(A2 - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
def test_k_cycle_matches_oracle(setting, prec, tol):
    from paper_2004_08146_gb300 import qcd
    dt = np.complex128 if prec == 0 else np.complex64
    b = synth.spinor(DIMS, 58, nvec=1)
    tau = [0.07]
    ref = setting["h"].cycle(b[0], tau[0])
    x = dev(b, dt)
    setting["ctx"].qcd_mg_cycle(qcd.QCD_OP_D, prec, 1, dev(b, dt), x, tau)
    assert relerr(host(x), ref) < tol


@pytest.mark.parametrize("precision", [0, 1])
def test_shifted_solve_with_k_cycle(setting, precision):
    """(Q - tau) x = b to 1e-10 (Eq. 1.1) with the three-level preconditioner
    at the Table 2 tolerances; the residual is measured by the oracle."""
    from paper_2004_08146_gb300 import qcd
    torch = torch_cuda()
    op = setting["op"]
    ctx = make_ctx(setting["U"], DIMS, setting["m0"], setting["csw"], sap_block=BLOCK, precision=precision,
                   levels=3, nv2=NV2, agg2=AGG2)
    ctx.qcd_mg_setup(NV, BLOCK)
    b = synth.spinor(DIMS, 59)
    x = torch.zeros(b.size, dtype=torch.complex128, device="cuda")
    rc, info = ctx.qcd_shifted_solve(dev(b), x, 0.1, 1e-10)
    assert rc == qcd.QCD_OK
    xs = host(x).reshape(DIMS + (4, 3))
    assert np.linalg.norm(op.Q_shift(xs, 0.1) - b) <= 1e-9 * np.linalg.norm(b)
