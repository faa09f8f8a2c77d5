"""Plain FP64 CPU oracle for the DPG multigrid (DPG-MG) solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything from this package.  The
product path (the CUDA library and its Python binding) never calls it, and it
never calls the product path: the two share no code.

What it computes follows Badger, Henneking, Petrides, Demkowicz, "Scalable DPG
Multigrid Solver for Helmholtz Problems: A Study on Convergence" (arXiv
2304.01728):

* ``basis``     1D Legendre / integrated-Legendre bases and Gauss rules
                (the exact-sequence spaces of Sec. 2, hexahedra only).
* ``mesh``      structured hexahedral meshes and the documented global
                trace-DOF numbering.
* ``element``   element Gram matrix of the adjoint graph norm (Eq. Gnorm),
                the ultraweak forms b, b-hat and the load (Sec. 2, Eq.
                variational-formulation), the DPG element matrix
                B^* G^{-1} B (Sec. 1.2 / Sec. 2 optimal test functions) and
                static condensation of the field DOFs (Sec. 1.2).
* ``hierarchy`` the DPG-MG level hierarchy of Sec. 3: p-injection, macro-grid
                condensation and natural inclusion (Sec. 3 "Prolongation"),
                coarse operators by restriction (Sec. 3 "Alternative
                construction"), vertex-patch additive Schwarz (Sec. 3
                "V-cycle and smoother").
* ``solver``    the V-cycle and MG-preconditioned conjugate gradients with the
                stopping rule of Sec. 4.
* ``problem``   sources and loads (Gaussian source, plane wave, manufactured
                polynomial solution) in the notation of Eq. helmholtz.

Every function is written for readability, not speed: dense numpy linear
algebra per element / per patch, Python loops over elements and patches.

Parity status.  All functions here are pinned by ``tests/test_oracle_*.py``
(closed forms, manufactured-solution exactness, plane-wave convergence rates,
HPD invariants, brute-force dense solves, block-elimination identities,
V-cycle symmetry).  Parity unpinned: the absolute PCG iteration counts (the
paper prints none; its figures are not available), and the effect of the
silent-point readings (patch rule at the boundary, damping, coarsest solve) on
them.
"""
