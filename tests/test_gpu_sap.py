"""SAP sweeps (Eq. 2.10) through the C ABI against the oracle's ``mg.SAP`` for
every kernel family the block size selects: 8-site blocks and 4^4 = 256-site
blocks (one thread per site, Krylov vectors in global scratch), 16-site
blocks (two lanes per site, one warp per block) and 32-site blocks (one warp
per block).  Fixed block-GMRES step counts (tolerance 0 in the oracle, a
negative tolerance in the library) make the iterates comparable step by
step, in both forms of the shifted operator, D - tau Gamma5 (Eq. 3.7) and
Q - tau (Eq. 3.6).  FP64 agrees to rounding (1e-10 relative), FP32 to 1e-4."""
import numpy as np
import pytest

from oracle.dirac import WilsonClover
from oracle import mg
from paper_2004_08146_gb300 import synth
from gpu_util import make_ctx, dev, host, relerr, torch_cuda

pytestmark = pytest.mark.gpu

ITERS = 4
CASES = [((8, 4, 4, 4), (2, 2, 2, 1)),     # 8 sites: block kernel
         ((8, 4, 4, 4), (2, 2, 2, 2)),     # 16 sites: chirality-split warp kernel
         ((8, 4, 4, 4), (4, 2, 2, 2)),     # 32 sites: warp kernel
         ((8, 8, 8, 8), (4, 4, 4, 4))]     # 256 sites: block kernel (the 4^4 blocks)


@pytest.mark.parametrize("dims,block", CASES)
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
def test_sap_block_families_match_oracle(dims, block, prec, tol):
    from paper_2004_08146_gb300 import qcd
    torch_cuda()
    U = synth.gauge_field(dims, 0.5, 71)
    m0, csw = -0.3, 1.3
    op = WilsonClover(U, m0, csw)
    ctx = make_ctx(U, dims, m0, csw, sap_block=block, sap_block_iters=ITERS)
    dt = np.complex128 if prec == 0 else np.complex64
    b = synth.spinor(dims, 72, nvec=2)
    x0 = synth.spinor(dims, 73, nvec=2)
    taus = [0.1, -0.2]
    sap = mg.SAP(dims, block, block_iters=ITERS, block_tol=0.0)
    for opc, form in ((qcd.QCD_OP_D, 'g5'), (qcd.QCD_OP_Q, 'Q')):
        xd = dev(x0, dt)
        ctx.qcd_sap(opc, prec, 2, dev(b, dt), xd, taus, 2, -1.0)
        got = host(xd).reshape((2,) + dims + (4, 3))
        for j in range(2):
            A = lambda v, t=taus[j]: mg.fine_apply(op, v, t, form)
            ref = sap.smooth(A, b[j], x0[j], 2)
            assert relerr(got[j], ref) < tol, (form, j)
    ctx.close()


def test_sap_fp16_basis_matches_oracle():
    """FP32 SAP on 16-site blocks with the block Krylov basis stored in FP16
    (params.sap_half): the sweeps follow the oracle's at fixed block-GMRES steps
    to the accuracy FP16 storage allows (5e-3 relative), both forms."""
    from paper_2004_08146_gb300 import qcd
    torch_cuda()
    dims, block = (8, 4, 4, 4), (2, 2, 2, 2)
    U = synth.gauge_field(dims, 0.5, 71)
    m0, csw = -0.3, 1.3
    op = WilsonClover(U, m0, csw)
    ctx = make_ctx(U, dims, m0, csw, sap_block=block, sap_block_iters=ITERS, sap_half=1)
    b = synth.spinor(dims, 72, nvec=2)
    x0 = synth.spinor(dims, 73, nvec=2)
    taus = [0.1, -0.2]
    sap = mg.SAP(dims, block, block_iters=ITERS, block_tol=0.0)
    qcd.qcd_stats_reset(0)
    for opc, form in ((qcd.QCD_OP_D, 'g5'), (qcd.QCD_OP_Q, 'Q')):
        xd = dev(x0, np.complex64)
        ctx.qcd_sap(opc, 1, 2, dev(b, np.complex64), xd, taus, 2, -1.0)
        got = host(xd).reshape((2,) + dims + (4, 3))
        for j in range(2):
            A = lambda v, t=taus[j]: mg.fine_apply(op, v, t, form)
            ref = sap.smooth(A, b[j], x0[j], 2)
            assert relerr(got[j], ref) < 5e-3, (form, j)
    # the FP16-basis kernel is the one that ran
    names = {r["name"]: r["launches"] for r in qcd.qcd_stats_read()}
    assert names.get("sap_block_f32h", 0) == 8 and "sap_block_f32" not in names
    ctx.close()


@pytest.mark.parametrize("prec,half,tol", [(0, 0, 1e-10), (1, 0, 1e-4), (1, 1, 5e-3)])
def test_sap_16site_blocks_many_rhs(prec, half, tol):
    """Six right-hand sides on 16-site blocks: four block solves share a CTA
    (one staged copy of the block's links and clover) and the last CTA holds
    two; every right-hand side follows the oracle's sweeps at fixed
    block-GMRES steps, both forms."""
    from paper_2004_08146_gb300 import qcd
    torch_cuda()
    dims, block, nrhs = (8, 4, 4, 4), (2, 2, 2, 2), 6
    U = synth.gauge_field(dims, 0.5, 75)
    m0, csw = -0.3, 1.3
    op = WilsonClover(U, m0, csw)
    ctx = make_ctx(U, dims, m0, csw, sap_block=block, sap_block_iters=ITERS, sap_half=half)
    dt = np.complex128 if prec == 0 else np.complex64
    b = synth.spinor(dims, 76, nvec=nrhs)
    x0 = synth.spinor(dims, 77, nvec=nrhs)
    taus = [0.05 * j - 0.12 for j in range(nrhs)]
    sap = mg.SAP(dims, block, block_iters=ITERS, block_tol=0.0)
    for opc, form in ((qcd.QCD_OP_D, 'g5'), (qcd.QCD_OP_Q, 'Q')):
        xd = dev(x0, dt)
        ctx.qcd_sap(opc, prec, nrhs, dev(b, dt), xd, taus, 2, -1.0)
        got = host(xd).reshape((nrhs,) + dims + (4, 3))
        for j in range(nrhs):
            A = lambda v, t=taus[j]: mg.fine_apply(op, v, t, form)
            ref = sap.smooth(A, b[j], x0[j], 2)
            assert relerr(got[j], ref) < tol, (form, j)
    ctx.close()
