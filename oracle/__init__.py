"""CPU oracle for the Lagrange-Legendre R-matrix hot path (TEST INFRASTRUCTURE).

Plain, slow, obviously-correct complex128 NumPy code written from the paper
(J. Lei, HPRMAT, arXiv 2512.11590) and the standard Lagrange-mesh formulas it
cites.  It shares no code with the GPU library: only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  The product path never calls it.

Modules
-------
mesh       Gauss-Legendre mesh on (0, a), basis values at a, kinetic+Bloch matrix.
system     dense C = T + L(0) + V - E and the surface right-hand sides Phi;
           dense and structured residuals.
lu         partial-pivoting LU (|Re|+|Im| pivot, first index on ties) and solves.
ddarith    double-double error-free transformations for the "truth" residual.
refine     FP64 LU + double-double-residual refinement ("truth" solution).
collision  R-matrix contraction and the collision matrix U (eta = 0).
pipeline   end-to-end oracle: problem -> X, R, U.

Pinning status (each function's docstring says what pins it; the tests under
``tests/test_oracle_*.py`` carry the pins).  No function is "parity unpinned".
"""
from . import mesh, system, lu, ddarith, refine, collision, pipeline  # noqa: F401
from .pipeline import oracle_solve  # noqa: F401
