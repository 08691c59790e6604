"""CPU FP64 oracle for the response-density-matrix solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA library (``paper_2009_03551_gb300``): no kernels, no helpers, no
constants.  The only common input is the seeded generator in ``synth``.

Contents (each function cites the paper passage it follows):

* ``dense``   - Oracle A, the exact definition: diagonalise H0, P0 from the
                occupied eigenvectors, P1 by the sum-over-states formula
                (Sec. 2.1, Eqs. DM1, CPSCF-U, epsilon1, cpscf-LCAO), and the
                polarizability (Eq. polar).
* ``lowdin``  - the non-orthogonal basis (Sec. 2.2): S^(-1/2) from the
                eigenpairs of S, the orthogonal-form Hamiltonians, Oracle A
                there, and the back-transform of P0 and P1.
* ``tc2``     - Oracle B, the algorithm step by step: Gershgorin bounds, the
                initial matrices, the TC2 recursion (Eq. TC2) coupled to the
                first-order recursion (Eq. TC2-CPSCF), block-norm truncation
                (the "filter" of Sec. 2.3) and the band-energy stopping rule.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
in ``tests/test_oracle_*.py`` (closed forms, invariants, finite differences,
scalar-map predictions).  Mixed-precision per-iteration trajectories are
parity unpinned (they are compared on limits and invariants only).
"""

from .dense import (  # noqa: F401
    exact_response,
    polarizability,
    projector_invariants,
    response_invariants,
)
from .lowdin import inverse_sqrt, lowdin_response  # noqa: F401
from .tc2 import (  # noqa: F401
    gershgorin_bounds,
    block_truncate,
    tc2_response,
    Tc2Result,
)
