"""Plain FP64 CPU oracle for the sparse-grid Krylov IIF DG method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never calls it and it never calls the CUDA library;
the two share no code, tables or constants.

Every function follows the paper (Liu, Cheng, Chen, Zhang, "Krylov implicit
integration factor discontinuous Galerkin methods on sparse grids for high
dimensional reaction-diffusion equations", arXiv:1810.11111) and cites the
section or equation it restates.  Arithmetic is numpy float64 throughout.

Modules
-------
basis      Legendre / Alpert multiwavelet bases (Section 2.1, eqs. sp4-sp9)
index_set  sparse-grid index set and coefficient layout (eqs. sp10-sp13)
operator   1D SIPG form in the hierarchical basis and the sparse-grid matvec
           (Section 2.1 bilinear form B, eq. sp3, Section 4 unidirectional
           principle)
projection L2 projection of separable initial data (Theorem 2.4, u_h(0)=Pu)
reaction   reaction term F(U) and its Jacobian by finest-grid Gauss quadrature
           (Section 4 implementation remarks, Section 5)
krylov     Arnoldi with re-orthogonalised Gram-Schmidt, Pade(13) expm with
           scaling and squaring, Krylov approximation of exp(dt A) v
           (eqs. krylov7-krylov8, Section 3); two extensions the paper does
           not have: Saad's (1992) a-posteriori error estimate and the
           exponential as a product of sub-projections
iif        Newton solve and the IIF2 time step (eq. krylov5, Example 3)
interp     the sparse-grid interpolation form of the reaction term (a
           deviation from the paper for its first stated future direction)
combination the combination-technique form of the reaction term (a second
           such deviation; no GPU counterpart yet)

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, library routines, invariants or printed paper values;
none is "parity unpinned" except the paper's Tables 1-2 digits, which the
oracle does not attempt to reproduce.
"""
