"""FP64 CPU oracle of the pressure-multigrid hot path (TEST INFRASTRUCTURE ONLY).

This package is the plain, slow reference that the CUDA library is checked against.  Only the
tests, the smoke check and the CPU-baseline leg of the benchmark may import it; the product
path (the C-ABI library and its Python binding) never does, and shares no code with it.

Every function cites the passage of Chen, Heaney, Gomes, Matar and Pain, "Solving the
discretised multiphase flow equations with interface capturing on structured grids using
machine learning libraries" (arXiv 2401.06755) that it follows.  Where the paper leaves a
detail open the reading taken is stated in the docstring.

Modules
  fem   - Q1 element integrals by Gauss quadrature, matrix-free assembled operators, and the
          generic filter application of Section 2.2.2.
  mg    - grid hierarchy, stencil apply (constant and variable coefficient), residual,
          restriction, prolongation, weighted Jacobi, coarsest solve, sawtooth V-cycle and
          the pressure solve.
  direct - dense LU and conjugate-gradient reference solvers (the exact solution of A x = b).
  flow  - explicit volume-fraction advection (Petrov-Galerkin, compressive), momentum
          predictor, pressure right-hand sides, velocity correction and the mass sum.

Parity status: every function is pinned by tests under ``tests/test_oracle_*.py`` against
closed forms, printed values, invariants or brute force, except where a docstring says
"parity unpinned".
"""
