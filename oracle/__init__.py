"""Plain FP64 CPU oracle for force-gradient Hybrid Monte Carlo on a 4D SU(3) lattice.

TEST INFRASTRUCTURE.  This package exists to check the CUDA path; it is not
part of the product.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import it.  It shares no code
with the CUDA library and imports nothing from the product package: inputs
are handed to it as plain numpy arrays.

Every function is a direct, slow, obviously-checkable statement of what the
paper (Kennedy, Clark, Silva, "Force Gradient Integrators", LAT2009) defines,
in float64/complex128, vectorised over lattice sites only.  Where the paper is
silent the oracle uses the standard convention listed next to the function.

Modules
  su3         -- Gell-Mann basis, exp(i c P), algebra projections (section 2)
  gauge       -- Wilson action, staple force, kinetic term (sections 2 and 4)
  integrators -- PQP, QPQ, PQPQP(alpha), Campostrini, force-gradient PQPQP
                 (section 3 and Table 1), HMC trajectory and Metropolis step
  fermion     -- Wilson-Dirac operator, even-odd preconditioning, CG and the
                 pseudofermion force (section 4, section 5)
  toy1d       -- one-dimensional anharmonic oscillator with closed-form
                 Poisson brackets, used to pin Table 1 shadow Hamiltonians

Parity status: every function is pinned by at least one test against a
closed form, an invariant, finite differences, a library routine or brute
force; see tests/test_oracle_*.py.  The displaced-force surrogate of the
force-gradient term has no Table 1 coefficient pin by design (it differs
from the exact force gradient at O(dt^5) per step); its order and its
agreement with the finite-difference exact force gradient are pinned.
"""
