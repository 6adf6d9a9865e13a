"""GPU parity of the Wilson-clover operator (Eq. 2.5 + clover, Eq. 3.6, 3.7)
against the FP64 oracle, through the C ABI.  FP64: 1e-13 relative (rounding
order only); FP32: 2e-6 relative (24-bit mantissa over ~50 terms per row)."""
import numpy as np
import pytest

from oracle.dirac import WilsonClover
from paper_2004_08146_gb300 import synth
from gpu_util import make_ctx, dev, host, relerr, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [((4, 4, 4, 4), 0.3, -0.2, 1.0, True),
         ((6, 4, 2, 4), 0.6, 0.1, 1.7, True),     # extent-2 direction: x+mu = x-mu
         ((2, 2, 2, 2), 0.5, -0.4, 1.3, False),   # smallest lattice, periodic time
         ((8, 6, 4, 2), 0.5, -0.1, 1.5, True)]


@pytest.mark.parametrize("dims,eps,m0,csw,antip", CASES)
def test_apply_Q_fp64(dims, eps, m0, csw, antip):
    from paper_2004_08146_gb300 import qcd
    U = synth.gauge_field(dims, eps, 11)
    op = WilsonClover(U, m0, csw, antiperiodic_t=antip)
    ctx = make_ctx(U, dims, m0, csw, antiperiodic_t=int(antip))
    psi = synth.spinor(dims, 12)
    x = dev(psi)
    y = x.clone()
    y.zero_()
    ctx.qcd_apply_Q(x, y, 0.37)
    assert relerr(host(y), op.Q_shift(psi, 0.37)) < 1e-13
    with pytest.raises(qcd.QcdError):
        ctx.qcd_apply_Q(x, x, 0.0)   # aliasing is rejected


@pytest.mark.parametrize("dims,eps,m0,csw,antip", CASES[:2])
@pytest.mark.parametrize("prec", [0, 1])
def test_apply_multi_rhs_both_forms(dims, eps, m0, csw, antip, prec):
    from paper_2004_08146_gb300 import qcd
    U = synth.gauge_field(dims, eps, 21)
    op = WilsonClover(U, m0, csw, antiperiodic_t=antip)
    ctx = make_ctx(U, dims, m0, csw, antiperiodic_t=int(antip))
    nrhs = 3
    psi = synth.spinor(dims, 22, nvec=nrhs)
    taus = [0.0, 0.21, -0.55]
    dt = np.complex128 if prec == 0 else np.complex64
    tol = 1e-13 if prec == 0 else 2e-6
    x = dev(psi, dt)
    for form in (qcd.QCD_OP_D, qcd.QCD_OP_Q):
        y = x.clone()
        ctx.qcd_apply(form, prec, nrhs, x, y, taus)
        got = host(y).reshape((nrhs,) + dims + (4, 3))
        for j in range(nrhs):
            ref = op.D_g5shift(psi[j], taus[j]) if form == qcd.QCD_OP_D else op.Q_shift(psi[j], taus[j])
            assert relerr(got[j], ref) < tol


def test_apply_c2_workload_full_field():
    """The 16 x 8^3 workload lattice (eps 0.5, csw 1.5), whole field, FP64 and FP32."""
    from paper_2004_08146_gb300 import qcd
    dims = (16, 8, 8, 8)
    U = synth.gauge_field(dims, 0.5, 1002)
    op = WilsonClover(U, -0.5, 1.5)
    ctx = make_ctx(U, dims, -0.5, 1.5)
    psi = synth.spinor(dims, 31)
    ref = op.D_g5shift(psi, 0.05)
    for prec, dt, tol in ((0, np.complex128, 1e-13), (1, np.complex64, 2e-6)):
        x = dev(psi, dt)
        y = x.clone()
        ctx.qcd_apply(qcd.QCD_OP_D, prec, 1, x, y, [0.05])
        assert relerr(host(y), ref) < tol


def test_hermiticity_on_gpu():
    """<x, Q y> = <Q x, y> (Eq. 2.7) evaluated with the GPU operator."""
    dims = (8, 4, 4, 4)
    U = synth.gauge_field(dims, 0.5, 41)
    ctx = make_ctx(U, dims, -0.3, 1.2)
    a, b = synth.spinor(dims, 42), synth.spinor(dims, 43)
    xa, xb = dev(a), dev(b)
    qa, qb = xa.clone(), xb.clone()
    ctx.qcd_apply_Q(xa, qa, 0.0)
    ctx.qcd_apply_Q(xb, qb, 0.0)
    l = np.vdot(a, host(qb))
    r = np.vdot(host(qa), b)
    assert abs(l - r) < 1e-13 * np.linalg.norm(a) * np.linalg.norm(host(qb))


@pytest.mark.parametrize("dims,nrhs", [((16, 8, 4, 4), 5), ((8, 8, 8, 8), 2), ((24, 8, 4, 4), 3)])
def test_apply_multi_rhs_time_bricks(dims, nrhs):
    """FP32 multi-right-hand-side applies on lattices whose site blocks are
    visited in bricks of 8 time slices (L1 L2 L3 a multiple of 128, L0 a
    multiple of 8): every site of every right-hand side against the oracle,
    both forms, 2e-6 relative."""
    from paper_2004_08146_gb300 import qcd
    U = synth.gauge_field(dims, 0.5, 41)
    op = WilsonClover(U, -0.3, 1.5)
    ctx = make_ctx(U, dims, -0.3, 1.5)
    psi = synth.spinor(dims, 42, nvec=nrhs)
    taus = [0.1 * j - 0.2 for j in range(nrhs)]
    x = dev(psi, np.complex64)
    for form in (qcd.QCD_OP_D, qcd.QCD_OP_Q):
        y = x.clone()
        y.zero_()
        ctx.qcd_apply(form, 1, nrhs, x, y, taus)
        got = host(y).reshape((nrhs,) + dims + (4, 3))
        for j in range(nrhs):
            ref = op.D_g5shift(psi[j], taus[j]) if form == qcd.QCD_OP_D else op.Q_shift(psi[j], taus[j])
            assert relerr(got[j], ref) < 2e-6, (form, j)
