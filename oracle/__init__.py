"""Plain FP64 CPU oracle for the GD-lambda-AMG hot path (arXiv 2004.08146).

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
restatement of what the GPU library computes, written from the paper in
numpy float64/complex128.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
CUDA product path never imports, links or executes anything in here, and this
package imports nothing from the product package.

Modules
-------
dirac   Wilson-clover operator D, Gamma5, Q = Gamma5 D (Sec. 2, Eq. 2.4, 2.5, 2.7);
        its derivative along su(3) link directions and the Hellmann-Feynman
        eigenvalue derivative (pinned by central differences)
mg      aggregation interpolation P, restriction P^H, Galerkin coarse operator
        D_c = P^H D P, SAP smoother, GMRES/FGMRES, the two-level cycle
        E_2g (Sec. 2, Eq. 2.8-2.11, Prop. 1), the three-level K-cycle and the
        local coherence measure (Sec. 3)
gd      generalized Davidson with harmonic (or Rayleigh-Ritz) extraction,
        thick restart, locking and interpolation updates (Sec. 3,
        Algorithm 1, Algorithm 2, Theorem 1, Eq. 3.4-3.6)

Every function cites the passage it restates.  Readings taken where the paper
is silent are stated in the function docstrings.
"""
