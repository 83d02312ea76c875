"""Plain FP64 CPU oracle of the SM-AMG preconditioned Wilson-Dirac solve.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check of the entry
module and the CPU-baseline leg of the benchmark may import or run anything in
this package; the library's compute path never does, and this package imports
nothing from the CUDA library or its Python binding.

Each function restates a step of the paper ("A first look at Structured-
Multiscale Algebraic Multigrid for Lattice Field Theory") in the paper's order
and notation, slowly and without blocking or fusion:

  wilson.py    the Wilson-Dirac operator D of Eq. (3) with the Pauli basis of
               Eq. (4), sigma_3 of Eq. (5) and the boundary conditions of Eq. (7)
  amg.py       wirebaskets with vertex/edge/interior roles (Sec. 4.1), the local
               interpolation of Eqs. (14)-(16), the global interpolator, the
               Galerkin product A_H = I_h^H A_h I_H^h (Sec. 2), the block
               Gauss-Seidel smoother, the coarsest direct solve and the V-cycle
               of Algorithm 1
  krylov.py    flexible GMRES (outer solver, Sec. 1 and Sec. 5)
  spectrum.py  critical mass from the spectrum of D (Sec. 5 and its
               critical-mass table)

Where the paper is silent or ambiguous the module docstrings state the reading
taken.  Every function is pinned by the "not gpu" tests to something other than
itself (closed forms, invariants, brute force, dense linear algebra).
"""
