"""The three-level hierarchy in the shape of the 64x32^3 workload -- 4^4
aggregates on the fine lattice, then 2^4 aggregates on the coarse lattice,
Nv = 24 (2 Nv = 48), nv2 = 8 -- on a 16^4 lattice the oracle builds in
seconds (level 1: 4^4 sites, level 2: 2^4 sites).  Through the C ABI against
the oracle's ``ThreeLevelMG``: P, the level-1 stencil, P2 and the level-2
stencil element by element (1e-12), and one K-cycle at fixed iteration
counts (FP64 1e-10, FP32 1e-4)."""
import numpy as np
import pytest

from oracle.dirac import WilsonClover
from oracle import mg
from paper_2004_08146_gb300 import synth
from gpu_util import make_ctx, dev, host, relerr, torch_cuda

pytestmark = pytest.mark.gpu

DIMS = (16, 16, 16, 16)
AGG, AGG2, SAP = (4, 4, 4, 4), (2, 2, 2, 2), (2, 2, 2, 2)
NV, NV2 = 24, 8
KC = dict(coarse_tol=0.0, coarse_maxiter=4, nu=2, sap_block_iters=4, gmres_smooth_iters=3, nu2=2)


@pytest.fixture(scope="module")
def setting():
    torch_cuda()
    U = synth.gauge_field(DIMS, 0.6, 161)
    m0, csw = -0.5, 1.9
    op = WilsonClover(U, m0, csw)
    vecs = synth.spinor(DIMS, 162, nvec=NV)
    h = mg.ThreeLevelMG(op, AGG, AGG2, SAP, NV, NV2, nu2=KC["nu2"], smooth2_iters=KC["gmres_smooth_iters"],
                        coarse2_tol=0.0, coarse2_maxiter=KC["coarse_maxiter"], nu=KC["nu"], coarse_tol=0.0,
                        coarse_maxiter=KC["coarse_maxiter"], smoother='sap', sap_block_iters=KC["sap_block_iters"],
                        sap_block_tol=0.0)
    h.set_vectors(vecs)
    ctx = make_ctx(U, DIMS, m0, csw, sap_block=SAP, sap_block_tol=-1.0, precision=0, levels=3, nv2=NV2,
                   agg2=AGG2, setup_iters=1, **KC)
    ctx.qcd_mg_setup(NV, AGG)                    # fixes the aggregate shape
    ctx.qcd_mg_update_from_eigvecs(dev(vecs), NV)
    b = synth.spinor(DIMS, 168, nvec=1)
    ref = h.cycle(b[0], 0.05)
    return dict(U=U, op=op, vecs=vecs, h=h, ctx=ctx, b=b, ref=ref)


def test_sizes(setting):
    info = setting["ctx"].qcd_mg_info2()
    assert info["dims"] == (2, 2, 2, 2) and info["nv2"] == NV2 and info["nv1"] == NV
    assert info["aggregate_sites"] == 16 and info["sites"] == 16


def test_interpolations_and_stencils_match_oracle(setting):
    ctx, h = setting["ctx"], setting["h"]
    assert relerr(ctx.qcd_mg_get_P(), h.interp.P) < 1e-12
    A = ctx.qcd_mg_get_coarse()
    assert np.max(np.abs(A - h.coarse.A)) < 1e-12 * np.max(np.abs(h.coarse.A))
    assert relerr(ctx.qcd_mg_get_P2(), h.interp2.P) < 1e-12
    A2 = ctx.qcd_mg_get_coarse2()
    assert np.max(np.abs(A2 - h.coarse2.A)) < 1e-12 * np.max(np.abs(h.coarse2.A))


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
def test_k_cycle_matches_oracle(setting, prec, tol):
    from paper_2004_08146_gb300 import qcd
    dt = np.complex128 if prec == 0 else np.complex64
    b = setting["b"]
    x = dev(b, dt)
    setting["ctx"].qcd_mg_cycle(qcd.QCD_OP_D, prec, 1, dev(b, dt), x, [0.05])
    assert relerr(host(x), setting["ref"]) < tol
