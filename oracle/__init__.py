"""FP64 CPU oracle of the LBM-RANS wall-function method (Ponsin & Lozano).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
reference against which the CUDA library is checked.  Only the test suite, the
package's ``smoke()`` entry and the CPU-baseline leg of the benchmark may import
it.  The product path never calls it, and it shares no code with the CUDA
library: it re-derives every formula from the paper in numpy float64.

Modules
-------
lattice  -- D2Q9 / D3Q19 velocity sets, equilibrium, Guo forcing, collisions
            (Section 2.1, Eqs. 1-8)
wallfn   -- SA-consistent wall function (Eqs. 15-16), log law, u_tau inversion
sa       -- Spalart-Allmaras model and its finite-difference discretisation
            (Section 2.2, Eqs. 10-14)
solver   -- the step in the paper's order: SA update, wall pre-pass, streaming,
            face conditions, regularized (HRFD) wall reconstruction, moments,
            collision (Sections 2-3, Eqs. 1-35)

Parity status of each function is stated in its docstring; "parity unpinned"
marks a function without an independent pin.
"""
from . import bounce, lattice, wallfn, sa, solver  # noqa: F401
from .solver import Oracle  # noqa: F401
