"""Plain FP64 CPU oracle for the distillation subtraction estimator.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import or call anything in this package; the GPU library never does, and
this package imports nothing from the GPU library.  The only code both sides share is the
seeded input generator ``lqcd_inputs`` (random numbers and field shapes, no method arithmetic).

Everything here is written from the definitions of "Subtraction method for disconnected
diagrams in full QCD" (Barca, Crawford, Finkenrath, Schaefer, Urrea-Nino), in numpy float64 /
complex128, with no blocking, fusion or reordering beyond what the definitions state:

* ``gamma``   Euclidean chiral gamma matrices, the 16-element Clifford table, Gamma-tilde (Sec. 2).
* ``dirac``   site indexing, even-odd and domain tables, clover-improved Wilson operator D,
              its adjoint, the Dirichlet domain operator D_Lambda (Sec. 2.1), dense D.
* ``solve``   CG on the normal equations and dense LU solves.
* ``smear``   spatial APE smearing with the polar-factor SU(3) projection (Sec. 3.1 smeared links).
* ``distill`` covariant 3D Laplacian eigenvectors, distillation sources, perambulators
              tau = V^dagger D^{-1} V, quark loops (Sec. 2, Sec. 3.1-3.2) and the full,
              completely factorised and subtracted disconnected correlators (Eqs. Cdisc,
              correlator_factorised, subtracted_correlator, corr1-corr4).

Parity status of every function is recorded in its module docstring; nothing on the hot path
is unpinned (see tests/test_oracle_*.py for the pins).
"""
