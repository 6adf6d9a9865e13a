"""The small projected eigenproblem of a Davidson step through the C ABI
(qcd_projected_eig, the kernels of qcd_eigs: Cholesky, FP32 Jacobi, FP64
refinement) against the oracle's ``gd.harmonic_ritz`` (Theorem 1, Eq. 3.5)
and ``gd.rayleigh_ritz`` (the Ritz-Galerkin condition of Sec. 3), for basis
sizes up to the library's cap of 112.  V: seeded random orthonormal basis of
the 4^4 workload's space; W = Q V with the oracle operator.

Bars: eigenvalues (1/theta for the harmonic pencil, theta for Rayleigh-Ritz)
within 1e-11 of the largest; each pair's coefficient vector agrees with the
oracle's up to a phase, |s_gpu^H G s_ref| >= 1 - 1e-8, wherever the pair is
separated from its neighbours by more than 1e-3 of the spectral radius."""
import numpy as np
import pytest

from oracle.dirac import WilsonClover
from oracle import gd
from paper_2004_08146_gb300 import synth
from gpu_util import make_ctx, torch_cuda

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)


@pytest.fixture(scope="module")
def basis():
    torch_cuda()
    U = synth.gauge_field(DIMS, 0.3, 1001)
    op = WilsonClover(U, -0.2, 1.0)
    m = 112
    X = synth.complex_gaussian((m, op.n), 81)
    V, _ = np.linalg.qr(X.T)
    W = np.stack([op.Q(V[:, j].reshape(DIMS + (4, 3))).reshape(-1) for j in range(m)], axis=1)
    return U, V, W


def _separated(ev, j, frac=1e-3):
    scale = np.max(np.abs(ev))
    d = np.abs(ev - ev[j])
    d[j] = np.inf
    return d.min() > frac * scale


@pytest.mark.parametrize("m", [20, 66, 112])
@pytest.mark.parametrize("extraction", [0, 1])
def test_projected_eig_matches_oracle(basis, m, extraction):
    U, V0, W0 = basis
    V, W = V0[:, :m], W0[:, :m]
    ctx = make_ctx(U, DIMS, -0.2, 1.0)
    G = W.conj().T @ W
    H = W.conj().T @ V
    if extraction == 0:
        th_ref, S_ref = gd.harmonic_ritz(V, W)
        th, S = ctx.qcd_projected_eig(G, H, 0)
        ev, ev_ref, M = 1.0 / th, 1.0 / th_ref, G
    else:
        th_ref, S_ref = gd.rayleigh_ritz(V, W)
        th, S = ctx.qcd_projected_eig(None, H, 1)
        ev, ev_ref, M = th, th_ref, np.eye(m)
    ctx.close()
    assert np.max(np.abs(ev - ev_ref)) <= 1e-11 * np.max(np.abs(ev_ref))
    # normalisation S^H G S = I (S^H S = I for Rayleigh-Ritz)
    assert np.max(np.abs(S.conj().T @ M @ S - np.eye(m))) < 1e-9
    checked = 0
    for j in range(m):
        if not _separated(ev_ref, j):
            continue
        ov = abs(np.vdot(S[:, j], M @ S_ref[:, j]))
        assert ov >= 1 - 1e-8, (j, ov)
        checked += 1
    assert checked >= m // 2
