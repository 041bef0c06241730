"""CPU FP64 oracle for the stochastic Magnus solver of the kinetic Langevin SPDE.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, deliberately
unoptimised restatement of the method of Kamm, Pagliarani & Pascucci,
"Numerical solution of kinetic SPDEs via stochastic Magnus expansion"
(arXiv 2207.09776).  It exists to check the CUDA path; only the test suite,
the smoke check and the bench's CPU-baseline leg may import it.  It shares no
code, table or constant generator with the CUDA library.

Modules
  philox        Philox4x32-10 counter-based generator + Box-Muller normals
  brownian      fine Brownian increments and the per-step iterated integrals
  discretization grids, finite-difference matrices, Kronecker assembly of B, A
  magnus        Magnus logarithms m1/m2/m3 and the iterated scheme
  euler         Euler-Maruyama comparator
  explicit      closed-form Gaussian solution (constant and time-dependent)
  errors        ME / AME / Err error norms and per-path moments

Parity notes.  Every function is pinned by a test in tests/test_oracle_*.py
against something other than itself (closed forms, brute force, published
known-answer vectors, invariants).  The one function without such a pin is
stated in its own docstring ("parity unpinned").
"""
