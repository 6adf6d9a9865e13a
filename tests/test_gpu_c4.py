"""GPU eigensolver on the 64 x 32^3 workload at full size (2,097,152 sites,
25,165,824 unknowns) in the configuration bench.py times (three-level MG:
4^4 then 2^4 aggregates, Nv = nv2 = 24; 16 targets per outer iteration,
m_min 30, m_max 50; FP16-stored SAP block basis; mixed precision), for the 4
smallest |lambda|, checked by properties that hold at any size:
* the run converges, |lambda| ascending, V^H V = I to 1e-9 (on the device);
* every returned pair is certified by the oracle's FP64 operator on the full
  lattice: ||Q v - lambda v|| <= 1e-8 and lambda = v^H Q v to 1e-10 relative
  (so each lambda lies within 1e-8 of an eigenvalue of Q, Weyl)."""
import numpy as np
import pytest

from oracle.dirac import WilsonClover
from paper_2004_08146_gb300 import synth, workloads
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def test_c4_smallest_pairs_certified():
    torch = torch_cuda()
    import bench
    from paper_2004_08146_gb300 import qcd
    w = workloads.get("c4_64x32c3")
    assert w["levels"] == 3 and w["block"] == 16
    dims, k = tuple(w["dims"]), 4
    U = synth.gauge_field(dims, w["eps"], w["seed"])
    n = 12 * int(np.prod(dims))
    ctx = qcd.Context(params=bench.workload_params(qcd, w, max_outer=2000),
                      stream=torch.cuda.current_stream().cuda_stream)
    ctx.qcd_set_gauge(U, dims, w["m0"], w["csw"])
    ctx.qcd_mg_setup(w["nv"], w["agg"])
    V = torch.zeros(k * n, dtype=torch.complex128, device="cuda")
    rc, lam, info = ctx.qcd_eigs(k, 1e-8, V)
    torch.cuda.synchronize()
    ctx.close()
    assert rc == qcd.QCD_OK and info.converged and info.max_residual <= 1e-8
    assert np.all(np.diff(np.abs(lam)) >= 0)
    Vm = V.view(k, n)
    G = Vm.conj() @ Vm.T
    assert (G - torch.eye(k, dtype=G.dtype, device=G.device)).abs().max().item() < 1e-9
    Vh = Vm.cpu().numpy()
    del V, Vm, G
    op = WilsonClover(U, w["m0"], w["csw"])
    for j in range(k):
        v = Vh[j].reshape(dims + (4, 3))
        Qv = op.Q(v)
        rho = np.vdot(v, Qv).real
        assert abs(rho - lam[j]) <= 1e-10 * abs(lam[j]), j
        assert np.linalg.norm(Qv - lam[j] * v) <= 1e-8, j
