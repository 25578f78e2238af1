"""Plain FP64 CPU oracle of the stochastic-TDH action of W and of the Tamm-Dancoff matrix A.

This package is TEST INFRASTRUCTURE. It is slow on purpose and follows the paper step by step.
Only the test suite, the smoke check of the package entry and the CPU-baseline leg of the
benchmark may import or run it; the library's compute path never does. It shares no code with the
CUDA path: the only module both sides use is the seeded input generator `sbse_inputs`.

Modules:
  tdh   - Coulomb operator, stochastic coefficients, stochastic TDH W^pol (difference form and the
          literal two-set form), the K and D contractions, A and its lowest eigenvalues.
  rpa   - deterministic linear-response (Casida) evaluation of the same damped W^pol, used to pin
          the TDH engine on tiny grids.
"""
from . import rpa, tdh  # noqa: F401
