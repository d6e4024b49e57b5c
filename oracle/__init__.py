"""FP64 CPU oracle for the preconditioned FGMRES solve of the monolithic FSI
Jacobian (Sec. 4 of the paper: Alg. 2 block-LDU preconditioner, Alg. 3 solid
Schur solve, fluid Schur solve, AMG sub-solves; GMRES outer solver).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package:
it is used by ``tests/``, by ``__graft_entry__.smoke()`` and by ``bench.py``'s
CPU-baseline / reference legs.  It shares no code with the CUDA library; both
read the same seeded inputs from ``fsigen``.

Parity pins: see ``tests/test_oracle_*.py`` (1D Poisson closed form and Thomas
algorithm, dense LU on tiny systems, exact-sub-solve identity
P = (D+L) D^-1 (D+U), <= 3-iteration nilpotency bound, monotone residuals,
Givens least squares = lstsq).
"""
from .amg import AMGParams, Hierarchy, sa_setup, vcycle, chebyshev, rigid_body_modes, translations
from .fgmres import FGMRESResult, fgmres
from .precond import Blocks, BlockLDU, PrecondParams, pressure_schur, solid_schur
from .solve import OracleSolver

__all__ = ["AMGParams", "Hierarchy", "sa_setup", "vcycle", "chebyshev", "rigid_body_modes", "translations",
           "FGMRESResult", "fgmres", "Blocks", "BlockLDU", "PrecondParams", "pressure_schur", "solid_schur",
           "OracleSolver"]
