"""qcd_sap_static -- the SAP entry point for callers that cannot allocate
device memory while they run (an application that hands the library a fixed
memory budget up front, or a plugin whose host owns every allocation) --
against qcd_sap on the same inputs and against the oracle's SAP, two calls
in a row (the static scratch keeps the previous call's contents), for every
kernel family: 8-site and 256-site blocks (Krylov vectors in the static
scratch), 16-site and 32-site blocks (Krylov basis in shared memory).
Tolerances: against qcd_sap (same kernels) FP64 1e-13, FP32 2e-6; against
the oracle at fixed block-GMRES steps FP64 1e-10, FP32 1e-4.  The second
call must leave the device's free memory unchanged."""
import numpy as np
import pytest

from oracle.dirac import WilsonClover
from oracle import mg
from paper_2004_08146_gb300 import synth
from gpu_util import make_ctx, dev, host, relerr, torch_cuda

pytestmark = pytest.mark.gpu

ITERS = 4


@pytest.mark.parametrize("dims,block", [((8, 4, 4, 4), (2, 2, 2, 1)), ((8, 4, 4, 4), (2, 2, 2, 2)),
                                        ((8, 4, 4, 4), (4, 2, 2, 2)), ((8, 8, 8, 8), (4, 4, 4, 4))])
@pytest.mark.parametrize("prec", [0, 1])
def test_sap_static_matches_sap_and_oracle(dims, block, prec):
    from paper_2004_08146_gb300 import qcd
    torch = torch_cuda()
    U = synth.gauge_field(dims, 0.5, 61)
    m0, csw = -0.3, 1.3
    op = WilsonClover(U, m0, csw)
    ctx = make_ctx(U, dims, m0, csw, sap_block=block, sap_block_iters=ITERS)
    dt = np.complex128 if prec == 0 else np.complex64
    tol_same = 1e-13 if prec == 0 else 2e-6
    tol_oracle = 1e-10 if prec == 0 else 1e-4
    nrhs = 2
    taus = [0.05, -0.2]
    sap = mg.SAP(dims, block, block_iters=ITERS, block_tol=0.0)
    for call in range(2):                      # two calls in a row
        b = synth.spinor(dims, 62 + call, nvec=nrhs)
        x0 = synth.spinor(dims, 64 + call, nvec=nrhs)
        for opc, form in ((qcd.QCD_OP_D, 'g5'), (qcd.QCD_OP_Q, 'Q')):
            xa = dev(x0, dt)
            ctx.qcd_sap(opc, prec, nrhs, dev(b, dt), xa, taus, 2, -1.0)
            bd, xb = dev(b, dt), dev(x0, dt)
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            ctx.qcd_sap_static(opc, prec, nrhs, bd, xb, taus, 2, -1.0)
            free1 = torch.cuda.mem_get_info()[0]
            if call == 1:                      # the first call may load kernel modules
                assert free1 == free0
            got = host(xb)
            assert relerr(got, host(xa)) < tol_same
            got = got.reshape((nrhs,) + dims + (4, 3))
            for j in range(nrhs):
                A = lambda v, t=taus[j]: mg.fine_apply(op, v, t, form)
                ref = sap.smooth(A, b[j], x0[j], 2)
                assert relerr(got[j], ref) < tol_oracle, (form, j)
    ctx.close()


def test_sap_static_rejects_oversize():
    """Fields beyond the 64 MiB static array are refused with EINVAL."""
    from paper_2004_08146_gb300 import qcd
    torch = torch_cuda()
    dims = (16, 8, 8, 16)
    U = synth.gauge_field(dims, 0.5, 65)
    ctx = make_ctx(U, dims, -0.3, 1.3, sap_block=(2, 2, 2, 2))
    n = 12 * int(np.prod(dims))
    fld = torch.zeros(64 * n, dtype=torch.complex128, device="cuda")   # in-bounds inputs either way
    with pytest.raises(qcd.QcdError) as e:
        ctx.qcd_sap_static(qcd.QCD_OP_D, 0, 64, fld, fld.clone(), [0.0] * 64, 1, 0.1)
    assert e.value.code == qcd.QCD_EINVAL
    assert "64 MiB" in str(e.value)
    ctx.close()


def test_sap_static_counts_krylov_scratch():
    """8-site blocks keep their block-GMRES vectors in the static scratch: a
    problem whose residual fields fit in 64 MiB but whose Krylov vectors do
    not (16x8^3, FP64, 12 right-hand sides, 10 block steps: 19 MB of
    residuals, 104 MB of Krylov vectors) is refused before any launch."""
    from paper_2004_08146_gb300 import qcd
    torch = torch_cuda()
    dims = (16, 8, 8, 8)
    U = synth.gauge_field(dims, 0.5, 66)
    ctx = make_ctx(U, dims, -0.3, 1.3, sap_block=(2, 2, 2, 1), sap_block_iters=10)
    nrhs = 12
    n = 12 * int(np.prod(dims))
    assert n * nrhs * 16 < 64 << 20
    b = torch.zeros(nrhs * n, dtype=torch.complex128, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(qcd.QcdError) as e:
        ctx.qcd_sap_static(qcd.QCD_OP_D, 0, nrhs, b, x, [0.0] * nrhs, 1, 0.1)
    assert e.value.code == qcd.QCD_EINVAL
    ctx.close()
