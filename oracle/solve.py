"""Oracle driver: set up Alg. 2 on one monolithic system and solve it with
right-preconditioned FGMRES.  Test infrastructure only."""
from __future__ import annotations

import time

import numpy as np
import scipy.sparse as sp

from .fgmres import fgmres
from .precond import BlockLDU, PrecondParams


class OracleSolver:
    def __init__(self, rowptr, colind, vals, offsets, dim, solid_coords=None,
                 params: PrecondParams | None = None, exact: bool = False):
        n = int(offsets[5])
        self.A = sp.csr_matrix((np.asarray(vals), np.asarray(colind), np.asarray(rowptr)), shape=(n, n))
        t0 = time.perf_counter()
        self.P = BlockLDU(self.A, offsets, dim, solid_coords, params, exact=exact)
        self.setup_s = time.perf_counter() - t0

    @classmethod
    def from_system(cls, system, params=None, exact=False):
        return cls(system.rowptr, system.colind, system.vals, system.offsets, system.dim,
                   system.solid_coords, params, exact)

    def solve(self, b, tol=1e-8, restart=100, maxit=1000, x0=None, correct=None, accept=1.0):
        t0 = time.perf_counter()
        res = fgmres(lambda v: self.A @ v, self.P, np.asarray(b, np.float64), tol, restart, maxit, x0, correct,
                     accept)
        res.solve_s = time.perf_counter() - t0
        return res
