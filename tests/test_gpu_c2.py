"""GPU eigensolver on the full 16 x 8^3 workload (the bench configuration),
checked by properties that hold at any size (the oracle's dense eig does not
reach 98,304 unknowns):
* every returned pair is certified by the oracle's FP64 operator:
  ||Q v - lambda v|| <= 1e-8, lambda = v^H Q v to 1e-10 relative, V^H V = I;
* the FP64 and the mixed-precision runs return the same eigenvalues (1e-10
  relative), and a run with another seed (other setup and start vectors) and
  2 instead of the workload's 4 targets per outer iteration finds the same
  set -- the weak completeness check available at this size."""
import numpy as np
import pytest

from oracle.dirac import WilsonClover
from paper_2004_08146_gb300 import synth, workloads
from gpu_util import make_ctx, host, torch_cuda

pytestmark = pytest.mark.gpu

K = 50


@pytest.fixture(scope="module")
def c2():
    torch_cuda()
    w = workloads.get("c2_16x8c3")
    dims = tuple(w["dims"])
    U = synth.gauge_field(dims, w["eps"], w["seed"])
    op = WilsonClover(U, w["m0"], w["csw"])
    return w, dims, U, op


def _run(c2, precision, seed, block=None):
    torch = torch_cuda()
    w, dims, U, op = c2
    ctx = make_ctx(U, dims, w["m0"], w["csw"], precision=precision, seed=seed, sap_block=w["sap"],
                   block=w["block"] if block is None else block, coarse_maxiter=w["coarse_maxiter"])
    ctx.qcd_mg_setup(w["nv"], w["agg"])
    V = torch.zeros(K * op.n, dtype=torch.complex128, device="cuda")
    rc, lam, info = ctx.qcd_eigs(K, 1e-8, V)
    assert rc == 0 and info.converged
    return lam, host(V).reshape(K, -1), info


@pytest.fixture(scope="module")
def mixed(c2):
    return _run(c2, 1, 20200417)


def test_pairs_certified_by_oracle(c2, mixed):
    w, dims, U, op = c2
    lam, V, info = mixed
    assert np.all(np.diff(np.abs(lam)) >= 0)
    G = V.conj() @ V.T
    assert np.max(np.abs(G - np.eye(K))) < 1e-9
    for j in range(K):
        v = V[j].reshape(dims + (4, 3))
        Qv = op.Q(v)
        rho = np.vdot(v, Qv).real
        assert abs(rho - lam[j]) <= 1e-10 * abs(lam[j])
        assert np.linalg.norm(Qv - lam[j] * v) <= 1e-8


def test_fp64_and_mixed_agree(c2, mixed):
    lam64, _, _ = _run(c2, 0, 20200417)
    assert np.max(np.abs(lam64 - mixed[0]) / np.abs(mixed[0])) < 1e-10


def test_other_seed_same_set(c2, mixed):
    lam2, _, _ = _run(c2, 1, 777, block=2)
    assert np.max(np.abs(lam2 - mixed[0]) / np.abs(mixed[0])) < 1e-10
