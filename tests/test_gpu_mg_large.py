"""GPU parity of the multigrid kernels at the coarse sizes of the large
workloads (2 Nv = 40 and 48, the 32x16^3 and 64x32^3 configurations)
against the FP64 oracle through the C ABI: P and the Galerkin stencil
(Sec. 2 above Eq. 2.9, Eq. 2.8, 2.9) element by element, restriction and
prolongation, the coarse apply in both forms, and one two-level cycle at
fixed iteration counts with every data layout of the one-launch coarse
GMRES (stencil and basis in shared memory, basis only, basis in global
memory).  Bars as in the small-lattice tests: FP64 1e-10 after the Krylov
steps (1e-12/1e-13 for the direct pieces), FP32 1e-4 (2e-6)."""
import numpy as np
import pytest

from oracle.dirac import WilsonClover
from oracle import mg
from paper_2004_08146_gb300 import synth
from gpu_util import make_ctx, dev, host, relerr, torch_cuda

pytestmark = pytest.mark.gpu

DIMS = (8, 8, 8, 8)
SAP = (2, 2, 2, 2)
# (aggregate, Nv): 256 coarse sites with 2 Nv = 48, and 128 coarse sites with
# 2 Nv = 40 (one coarse site per CTA, so the FP32 stencil blocks fit in shared memory)
SHAPES = [((2, 2, 2, 2), 24), ((4, 2, 2, 2), 20)]
CYCLE = dict(coarse_maxiter=8, nu=2, sap_block_iters=4)


@pytest.fixture(scope="module", params=SHAPES, ids=["agg2222_nv24", "agg4222_nv20"])
def setting(request):
    torch_cuda()
    agg, nv = request.param
    U = synth.gauge_field(DIMS, 0.5, 151)
    m0, csw = -0.3, 1.3
    op = WilsonClover(U, m0, csw)
    vecs = synth.spinor(DIMS, 152, nvec=nv)
    h = mg.TwoLevelMG(op, agg, SAP, nv, nu=CYCLE["nu"], coarse_tol=0.0, coarse_maxiter=CYCLE["coarse_maxiter"],
                      smoother='sap', sap_block_iters=CYCLE["sap_block_iters"], sap_block_tol=0.0)
    h.set_vectors(vecs)
    ctx = make_ctx(U, DIMS, m0, csw, sap_block=SAP, sap_block_tol=-1.0, coarse_tol=0.0, precision=0,
                   coarse_maxiter=CYCLE["coarse_maxiter"], nu=CYCLE["nu"], sap_block_iters=CYCLE["sap_block_iters"],
                   setup_iters=1)
    ctx.qcd_mg_setup(nv, agg)                    # fixes the aggregate shape
    ctx.qcd_mg_update_from_eigvecs(dev(vecs), nv)
    b = synth.spinor(DIMS, 158, nvec=1)
    ref = h.cycle(b[0], 0.07)
    return dict(U=U, op=op, vecs=vecs, h=h, ctx=ctx, m0=m0, csw=csw, agg=agg, nv=nv, b=b, cycle_ref=ref)


def test_P_and_stencil_match_oracle(setting):
    ctx, h = setting["ctx"], setting["h"]
    assert relerr(ctx.qcd_mg_get_P(), h.interp.P) < 1e-12
    A = ctx.qcd_mg_get_coarse()
    assert np.max(np.abs(A - h.coarse.A)) < 1e-12 * np.max(np.abs(h.coarse.A))


@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 2e-6)])
def test_restrict_prolong_apply(setting, prec, tol):
    from paper_2004_08146_gb300 import qcd
    torch = torch_cuda()
    ctx, h = setting["ctx"], setting["h"]
    dt = np.complex128 if prec == 0 else np.complex64
    tdt = torch.complex128 if prec == 0 else torch.complex64
    nrhs = 2
    info = ctx.qcd_mg_info()
    nco = info["coarse_sites"] * 2 * setting["nv"]
    r = synth.spinor(DIMS, 153, nvec=nrhs)
    xc = torch.zeros(nrhs * nco, dtype=tdt, device="cuda")
    ctx.qcd_mg_restrict(prec, nrhs, dev(r, dt), xc)
    got = host(xc).reshape(nrhs, -1)
    for j in range(nrhs):
        assert relerr(got[j], h.interp.restrict(r[j]).reshape(-1)) < tol
    c = synth.complex_gaussian((nrhs, nco), 154)
    x = dev(r, dt)
    ctx.qcd_mg_prolong(prec, nrhs, dev(c, dt), x)
    got = host(x).reshape(nrhs, -1)
    for j in range(nrhs):
        assert relerr(got[j], h.interp.prolong(c[j]).reshape(-1)) < tol
    taus = [0.13, -0.4]
    for op, form in ((qcd.QCD_OP_D, 'g5'), (qcd.QCD_OP_Q, 'Q')):
        y = torch.zeros(nrhs * nco, dtype=tdt, device="cuda")
        ctx.qcd_coarse_apply(op, prec, nrhs, dev(c, dt), y, taus)
        got = host(y).reshape(nrhs, -1)
        for j in range(nrhs):
            # FP32 applies: 1e-5 (FMA units, bulk-copy staging); FP64: the FP64 tolerance
            assert relerr(got[j], h.coarse.apply(c[j], taus[j], form).reshape(-1)) < (tol if prec == 0 else 1e-5)


@pytest.mark.parametrize("tensor,offset,kernel,tol", [(0, 0, "coarse_apply_bulk", 2e-6),
                                                      (0, 1, "coarse_apply_f32", 2e-6),
                                                      (1, 0, "coarse_apply_tc", 1e-5)])
def test_coarse_apply_many_rhs_tensor_and_fma(setting, tensor, offset, kernel, tol):
    """The FP32 coarse stencil on 20 right-hand sides (two chunks of the
    multi-right-hand-side kernels), both forms, against the oracle's stencil:
    FMA units with the stencil blocks and vectors staged by bulk asynchronous
    copies (16-byte aligned vectors), FMA units with plain loads (vectors one
    complex64 off a 16-byte boundary), and tensor cores (3xTF32 split).  No
    bounded wait gives up."""
    from paper_2004_08146_gb300 import qcd
    torch = torch_cuda()
    ctx, h = setting["ctx"], setting["h"]
    ctx.qcd_set_params(qcd.default_params(sap_block=SAP, sap_block_tol=-1.0, coarse_tol=0.0, precision=0,
                                          setup_iters=1, coarse_tensor=tensor, **CYCLE))
    nrhs = 20
    info = ctx.qcd_mg_info()
    nco = info["coarse_sites"] * 2 * setting["nv"]
    c = synth.complex_gaussian((nrhs, nco), 155)
    taus = [0.01 * j - 0.1 for j in range(nrhs)]
    t0 = qcd.qcd_stats_wait_timeouts()
    qcd.qcd_stats_reset(1)
    for op, form in ((qcd.QCD_OP_D, 'g5'), (qcd.QCD_OP_Q, 'Q')):
        xin = torch.zeros(nrhs * nco + offset, dtype=torch.complex64, device="cuda")
        xin[offset:] = dev(c, np.complex64)
        y = torch.zeros(nrhs * nco, dtype=torch.complex64, device="cuda")
        ctx.qcd_coarse_apply(op, 1, nrhs, xin[offset:], y, taus)
        got = host(y).reshape(nrhs, -1)
        for j in range(nrhs):
            assert relerr(got[j], h.coarse.apply(c[j], taus[j], form).reshape(-1)) < tol, (form, j)
    names = {r["name"]: r["launches"] for r in qcd.qcd_stats_read()}
    assert names.get(kernel, 0) == 2, names
    assert qcd.qcd_stats_wait_timeouts() == t0
    ctx.qcd_set_params(qcd.default_params(sap_block=SAP, sap_block_tol=-1.0, coarse_tol=0.0, precision=0,
                                          setup_iters=1, **CYCLE))


@pytest.mark.parametrize("layout", [0, 1, 2, 3])
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
def test_two_level_cycle_every_coarse_layout(setting, layout, prec, tol):
    """One cycle with the coarse GMRES's data forced into each layout (a
    forced layout that does not fit is refused with EINVAL, and layout 1
    fits only in the FP32 run on 128 coarse sites)."""
    from paper_2004_08146_gb300 import qcd
    dt = np.complex128 if prec == 0 else np.complex64
    kw = dict(sap_block=SAP, sap_block_tol=-1.0, coarse_tol=0.0, precision=0, setup_iters=1, **CYCLE)
    ctx = make_ctx(setting["U"], DIMS, setting["m0"], setting["csw"], **kw)
    ctx.qcd_mg_setup(setting["nv"], setting["agg"])
    ctx.qcd_mg_update_from_eigvecs(dev(setting["vecs"]), setting["nv"])
    ctx.qcd_set_params(qcd.default_params(coarse_layout=layout, **kw))
    b = setting["b"]
    x = dev(b, dt)
    fits = layout != 1 or (prec == 1 and setting["agg"] == (4, 2, 2, 2))
    if not fits:
        with pytest.raises(qcd.QcdError) as e:
            ctx.qcd_mg_cycle(qcd.QCD_OP_D, prec, 1, dev(b, dt), x, [0.07])
        assert e.value.code == qcd.QCD_EINVAL
    else:
        ctx.qcd_mg_cycle(qcd.QCD_OP_D, prec, 1, dev(b, dt), x, [0.07])
        assert relerr(host(x), setting["cycle_ref"]) < tol
    ctx.close()
