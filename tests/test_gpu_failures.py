"""Failure paths of the C ABI on the GPU, all made on the host (no device
fault is provoked):
* qcd_set_gauge refuses links that are not SU(3) matrices (Sec. 2): a
  non-finite entry or a non-unitary link returns EINVAL and leaves no field;
* qcd_shifted_solve that cannot reach its tolerance returns ENOCONV with the
  best iterate in x and its true residual in info (measured here with the
  oracle operator);
* qcd_eigs stopped by its outer-iteration cap returns ENOCONV with the pairs
  it has locked (each within the tolerance, checked with the oracle
  operator) and NaN for the rest;
* a bounded device-side wait that runs out (an mbarrier nothing arrives at,
  ~1 ms limit) is counted and reported as ETIMEOUT, and the context keeps
  working."""
import numpy as np
import pytest

from oracle.dirac import WilsonClover
from paper_2004_08146_gb300 import synth
from gpu_util import make_ctx, dev, host, torch_cuda

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)


@pytest.mark.parametrize("bad", ["nan", "inf", "nonunitary"])
def test_set_gauge_rejects_non_su3_links(bad):
    from paper_2004_08146_gb300 import qcd
    torch = torch_cuda()
    U = synth.gauge_field(DIMS, 0.3, 91)
    if bad == "nan":
        U[1, 2, 3, 0, 2, 1, 0] = np.nan
    elif bad == "inf":
        U[0, 0, 0, 1, 3, 0, 2] = np.inf
    else:
        U[3, 1, 0, 2, 1] *= 1.01
    ctx = qcd.Context(stream=torch.cuda.current_stream().cuda_stream)
    with pytest.raises(qcd.QcdError) as e:
        ctx.qcd_set_gauge(U, DIMS, -0.2, 1.0)
    assert e.value.code == qcd.QCD_EINVAL
    # nothing was kept: operator calls report the missing field
    x = torch.zeros(12 * 256, dtype=torch.complex128, device="cuda")
    with pytest.raises(qcd.QcdError) as e2:
        ctx.qcd_apply_Q(x, torch.zeros_like(x), 0.0)
    assert e2.value.code == qcd.QCD_ENOTSETUP
    ctx.close()


def test_shifted_solve_enoconv_returns_best_iterate():
    from paper_2004_08146_gb300 import qcd
    torch = torch_cuda()
    U = synth.gauge_field(DIMS, 0.3, 1001)
    op = WilsonClover(U, -0.2, 1.0)
    ctx = make_ctx(U, DIMS, -0.2, 1.0, precision=1)
    ctx.qcd_mg_setup(8, (2, 2, 2, 2))
    b = synth.spinor(DIMS, 92)
    x = torch.zeros(b.size, dtype=torch.complex128, device="cuda")
    rc, info = ctx.qcd_shifted_solve(dev(b), x, 0.1, 1e-30)   # below FP64 round-off: unreachable
    assert rc == qcd.QCD_ENOCONV
    xs = host(x).reshape(DIMS + (4, 3))
    res = np.linalg.norm(b - op.Q_shift(xs, 0.1)) / np.linalg.norm(b)
    assert res < 1e-12                                       # the best iterate is a solution to round-off
    assert abs(info.residual - res) <= 1e-13 + 0.1 * res      # and info reports its residual
    assert info.refinements == 200
    ctx.close()


def test_eigs_enoconv_returns_locked_pairs():
    from paper_2004_08146_gb300 import qcd
    torch = torch_cuda()
    U = synth.gauge_field(DIMS, 0.3, 1001)
    op = WilsonClover(U, -0.2, 1.0)
    ctx = make_ctx(U, DIMS, -0.2, 1.0, precision=1, max_outer=6)
    ctx.qcd_mg_setup(8, (2, 2, 2, 2))
    k = 10
    V = torch.zeros(k * op.n, dtype=torch.complex128, device="cuda")
    rc, lam, info = ctx.qcd_eigs(k, 1e-8, V)
    assert rc == qcd.QCD_ENOCONV and not info.converged
    assert info.outer == 6 and info.locked < k
    got = min(info.locked, k)
    assert np.all(np.isnan(lam[got:]))
    Vh = host(V).reshape(k, -1)
    for j in range(got):
        v = Vh[j].reshape(DIMS + (4, 3))
        assert np.linalg.norm(op.Q(v) - lam[j] * v) <= 1e-8
    ctx.close()


def test_bounded_wait_runs_out_and_context_stays_usable():
    from paper_2004_08146_gb300 import qcd
    torch = torch_cuda()
    U = synth.gauge_field(DIMS, 0.3, 93)
    op = WilsonClover(U, -0.2, 1.0)
    ctx = make_ctx(U, DIMS, -0.2, 1.0)
    n0 = qcd.qcd_stats_wait_timeouts()
    assert ctx.qcd_selftest_wait_limit() == qcd.QCD_ETIMEOUT
    assert qcd.qcd_stats_wait_timeouts() == n0 + 1
    # the context still works, and later calls do not report the old timeout
    psi = synth.spinor(DIMS, 94)
    x = dev(psi)
    y = torch.zeros_like(x)
    ctx.qcd_apply_Q(x, y, 0.1)
    ref = op.Q_shift(psi, 0.1)
    assert np.linalg.norm(host(y).reshape(ref.shape) - ref) <= 1e-13 * np.linalg.norm(ref)
    ctx.qcd_mg_setup(8, (2, 2, 2, 2))
    xs = torch.zeros_like(x)
    rc, info = ctx.qcd_shifted_solve(x, xs, 0.05, 1e-8)
    assert rc == qcd.QCD_OK
    assert qcd.qcd_stats_wait_timeouts() == n0 + 1
