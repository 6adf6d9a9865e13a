"""qcd_sap_static -- the allocation-free SAP entry point for callers that
cannot allocate device memory while they run -- against qcd_sap on the same
inputs, two calls in a row (the static scratch keeps the previous call's
contents), for 16-site blocks (warp kernel) and 256-site blocks (Krylov
vectors in the static scratch).  Tolerances as in the other SAP parity tests:
FP64 1e-13, FP32 2e-6 relative (same kernels, so agreement is expected to be
exact up to the order of floating-point reductions)."""
import numpy as np
import pytest

from paper_2004_08146_gb300 import synth
from gpu_util import make_ctx, dev, host, relerr, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,block", [((8, 4, 4, 4), (2, 2, 2, 2)), ((8, 8, 8, 8), (4, 4, 4, 4))])
@pytest.mark.parametrize("prec", [0, 1])
def test_sap_static_matches_sap(dims, block, prec):
    from paper_2004_08146_gb300 import qcd
    torch_cuda()
    U = synth.gauge_field(dims, 0.5, 61)
    ctx = make_ctx(U, dims, -0.3, 1.3, sap_block=block, sap_block_iters=6)
    dt = np.complex128 if prec == 0 else np.complex64
    tol = 1e-13 if prec == 0 else 2e-6
    nrhs = 2
    taus = [0.05, -0.2]
    for call in range(2):                      # two calls in a row
        b = synth.spinor(dims, 62 + call, nvec=nrhs)
        x0 = synth.spinor(dims, 64 + call, nvec=nrhs)
        for op in (qcd.QCD_OP_D, qcd.QCD_OP_Q):
            xa = dev(x0, dt)
            ctx.qcd_sap(op, prec, nrhs, dev(b, dt), xa, taus, 2, 0.1)
            xb = dev(x0, dt)
            ctx.qcd_sap_static(op, prec, nrhs, dev(b, dt), xb, taus, 2, 0.1)
            assert relerr(host(xb), host(xa)) < tol


def test_sap_static_rejects_oversize():
    """Fields beyond the 64 MiB static array are refused with EINVAL."""
    from paper_2004_08146_gb300 import qcd
    torch = torch_cuda()
    dims = (16, 8, 8, 16)
    U = synth.gauge_field(dims, 0.5, 65)
    ctx = make_ctx(U, dims, -0.3, 1.3, sap_block=(2, 2, 2, 2))
    small = torch.zeros(16, dtype=torch.complex128, device="cuda")
    with pytest.raises(qcd.QcdError) as e:
        ctx.qcd_sap_static(qcd.QCD_OP_D, 0, 64, small, small, [0.0] * 64, 1, 0.1)
    assert e.value.code == qcd.QCD_EINVAL
    assert "64 MiB" in str(e.value)
