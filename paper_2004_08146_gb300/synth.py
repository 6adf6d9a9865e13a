"""Seeded synthetic inputs: SU(3) gauge links, spinors, su(3) directions.

This module only draws inputs; it holds none of the eigensolver's
arithmetic, so both the GPU tests and the CPU oracle tests take their inputs
from here.  The paper's gauge ensembles (Table 1: CLS-type and heat-bath
configurations) are not available; random links U = exp(i eps H) stand in
for them, with eps steering the roughness and therefore the conditioning.

Layouts follow the library's C ABI: lattice ``dims = (L0, L1, L2, L3)`` with
mu = 0 the time direction and mu = 3 the fastest site index,
links ``[L0, L1, L2, L3, mu, row, col]`` complex128,
spinors ``[L0, L1, L2, L3, spin, colour]`` complex128.
"""
import numpy as np


def _rng(seed):
    return np.random.default_rng(np.random.SeedSequence(int(seed)))


def traceless_hermitian(rng, shape):
    """Traceless Hermitian 3x3 matrices: H = (G + G^H)/2 - tr/3 with G having
    iid N(0,1) real and imaginary parts (off-diagonal entries of H then have
    E|h|^2 = 1, diagonal entries N(0,1) before the trace is removed)."""
    G = rng.standard_normal(shape + (3, 3)) + 1j * rng.standard_normal(shape + (3, 3))
    H = 0.5 * (G + np.conj(np.swapaxes(G, -1, -2)))
    tr = np.trace(H, axis1=-2, axis2=-1).real / 3.0
    H = H - tr[..., None, None] * np.eye(3)
    return H


def _expi_hermitian(H, eps):
    """exp(i eps H) for Hermitian H through its eigendecomposition."""
    w, Vec = np.linalg.eigh(H)
    ph = np.exp(1j * eps * w)
    return (Vec * ph[..., None, :]) @ np.conj(np.swapaxes(Vec, -1, -2))


def reunitarize(U):
    """Project onto SU(3): Gram-Schmidt on rows 0 and 1, row 2 = conj(r0 x r1)."""
    U = np.array(U, dtype=np.complex128, copy=True)
    r0 = U[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = U[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def gauge_field(dims, eps, seed):
    """Links U_mu(x) = exp(i eps H) (H traceless Hermitian, see above),
    re-unitarised; shape dims + (4, 3, 3)."""
    dims = tuple(int(d) for d in dims)
    rng = _rng(seed)
    H = traceless_hermitian(rng, dims + (4,))
    return reunitarize(_expi_hermitian(H, eps))


def unit_gauge(dims):
    """Free field U = 1."""
    dims = tuple(int(d) for d in dims)
    U = np.zeros(dims + (4, 3, 3), dtype=np.complex128)
    U[..., :, :, :] = np.eye(3)
    return U


def random_su3(dims, seed, eps=np.pi):
    """One SU(3) matrix per site (e.g. a gauge transformation Omega(x))."""
    dims = tuple(int(d) for d in dims)
    rng = _rng(seed)
    return reunitarize(_expi_hermitian(traceless_hermitian(rng, dims), eps))


def spinor(dims, seed, nvec=None):
    """Complex Gaussian spinor(s): Re, Im iid N(0,1); shape dims + (4, 3), or
    (nvec,) + dims + (4, 3)."""
    dims = tuple(int(d) for d in dims)
    rng = _rng(seed)
    shape = dims + (4, 3) if nvec is None else (int(nvec),) + dims + (4, 3)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def complex_gaussian(shape, seed):
    rng = _rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def su3_directions(dims, seed, ndir):
    """ndir random traceless Hermitian fields X_mu(x), shape (ndir,) + dims + (4, 3, 3)."""
    dims = tuple(int(d) for d in dims)
    rng = _rng(seed)
    return traceless_hermitian(rng, (int(ndir),) + dims + (4,))
