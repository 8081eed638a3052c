"""FP64 CPU oracle of the approximate Gauss-Newton gain solver (arxiv 2412.10072).

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package.  It shares no code with the CUDA
library in ``paper_2412_10072_gb300``: the solver arithmetic lives in
``qc_oracle.c`` (plain C, double precision); this package compiles it with
gcc and calls it through ctypes.

Parity status of each oracle function (what pins it, see ``tests/``):

- ``normal_equations``: pinned by finite-difference Wirtinger Jacobians on
  3-antenna cases for diagonal, full and phase-only terms, by the Hermitian
  positive-semidefinite invariant and by the StefCal closed form.
- ``solve``: pinned by exact recovery of the true gains (up to the gauge) on
  noise-free data, by the 3-antenna closure relations, and by chi^2 = 0 at the
  truth.
- ``residual``: pinned by chi^2 = 0 at the true gains on noise-free data and
  by the noise statistics of chi^2 on noisy data.
- delay terms (Scenario 2): pinned by a forward model written in the test,
  central differences of it in the four real parameters, the chi^2
  gradient, exact recovery of generating phases and delays, and the
  singular single-frequency case (``tests/test_oracle_delay.py``).
- ``delay_init`` (the delay term's initial estimate, Section 4.3): pinned by
  exact recovery of delays on the transform's grid (the triangle-inequality
  bound), off-grid delays within half a step, flagged cells left out, and a
  solve from the estimate reaching delays a zero start cannot
  (``tests/test_oracle_delay_init.py``).
- ``mad_flag`` (MAD residual flagging): pinned by order statistics against
  a sort, planted outliers, the Gaussian spread of the MAD and the
  exclusion of flagged samples (``tests/test_oracle_mad.py``).
- ``moments`` (sufficient-statistics pre-reduction of a single diagonal
  term): its normal equations and chi^2 equal the sample-by-sample ones
  (``tests/test_oracle_moments.py``).
- ``dd`` (direction-dependent chains, N_D >= 1): pinned by the one-direction
  C oracle, Wirtinger finite differences with two directions for
  direction-dependent and direction-independent solved terms, and exact
  recovery of direction-dependent gains (``tests/test_oracle_dd.py``).
- ``mlp``: pinned by central finite differences of its own loss.
"""
from .oracle import (OC_DIAG, OC_FULL, OC_PHASE, OC_DELAY, OracleProblem, OracleTerm, build,  # noqa: F401
                     normal_equations, residual, solve, solve_term, block_solve)
from .gauge import reference_diag, reference_chain, chain_products  # noqa: F401
from .delay_init import delay_init  # noqa: F401
from .mad_flag import mad_flag  # noqa: F401
