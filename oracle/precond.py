"""Approximate block-LDU preconditioner of Sec. 4 (Alg. 2) with the solid Schur
solve of Sec. 4.3 (Alg. 3) and the fluid Schur solve of Sec. 4.4.  Oracle copy:
plain scipy, FP64, test infrastructure only.

Block structure (Eq. mat:small): rows/columns in the order m | s | f with
s = (s_v, s_u) and f = (f_v, f_p):
    A = [[M, C_ms, 0], [C_sm, S, C_sf], [C_fm, C_fs, F]].
Alg. 2 (C_sm dropped, Schur perturbation ignored, Sec. 4.1):
    x_m = M^-1 r_m;  x_s = S^-1 r_s;  x_f = F^-1 (r_f - C_fm x_m - C_fs x_s);
    x_s -= S^-1 C_sf x_f;  x_m -= M^-1 C_ms x_s.
Alg. 3 (Sec. 4.3) with S = [[A_vv, A_vu], [A_uv, A_uu]], A_uu the solid mass
matrix and A_uv = -dt*theta*A_uu on its free rows (no entries on fixed rows):
    y = A_uu^-1 r_u;  x_v = S_hat^-1 (r_v - A_vu y),  S_hat = A_vv + dt*theta*A_vu;
    x_u = A_uu^-1 (r_u - A_uv x_v) = y + dt*theta x_v on the free rows, y on fixed rows
(the second solve of Alg. 3 written out with A_uu^-1 A_uu = I: one mass solve
serves both steps).
Fluid (Sec. 4.4, "the same Schur-complement approach as for the solid"; the
reading taken here is the SIMPLE-type pressure Schur approximation):
    y_v = A_ff^-1 r_v;  x_p = S_p^-1 (r_p - B_pv y_v);  x_v = A_ff^-1 (r_v - B_vp x_p),
    S_p = C_pp - B_pv diag(A_ff)^-1 B_vp.
With fluid_gmres_iters = k > 0 each A_ff^-1 above is k steps of GMRES on A_ff,
right-preconditioned by the A_ff V-cycle(s), from a zero start (Sec. 4.4: an
AMG-preconditioned GMRES approximates the fluid inverses); k is fixed (no
stopping test), and the map r -> x is then nonlinear in r, which the outer
flexible GMRES allows.
Every inverse is a fixed number of smoothed-aggregation V-cycles (``amg.py``,
x <- x + V(r - A x) after the first); A_uu^-1 is a Chebyshev-Jacobi polynomial
(Chebyshev semi-iteration for mass matrices, Wathen & Rees, ETNA 34, 2009).  ``exact=True`` replaces all of them by sparse LU
solves, which turns Alg. 2 into P^-1 r with P = (D + L) D^-1 (D + U),
D = diag(M, S, F), L/U the strict block triangles of A with C_sm = 0.
Other block factorisations (the remark after Sec. 4.1: the LDU form depends on the
block ordering, and other orderings give other preconditioners), chosen by
``variant``: "lower" applies (D + L)^-1 (Alg. 2 steps 1-3), "upper" (D + U)^-1
(x_f = F^-1 r_f, x_s = S^-1 (r_s - C_sf x_f), x_m = M^-1 (r_m - C_ms x_s)) and
"diag" D^-1, each with the same approximate inverses.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .amg import AMGParams, chebyshev, point_dinv, power_lambda, rigid_body_modes, sa_setup, translations, vcycle
from .fgmres import fgmres


@dataclass
class PrecondParams:
    amg: AMGParams = field(default_factory=AMGParams)
    dt_theta: float = 0.01         # c = dt * theta of the solid Schur complement
    mass_degree: int = 12          # Chebyshev degree of the solid mass solve
    mass_ratio: float = 8.0        # its interval [lambda/mass_ratio, cheb_upper*lambda]
    vcycles_mesh: int = 1          # V-cycles per application of M^-1
    vcycles_solid: int = 2         # ... of S_hat^-1
    vcycles_fluid: int = 1         # ... of A_ff^-1
    vcycles_pressure: int = 1      # ... of S_p^-1
    fluid_gmres_iters: int = 0     # > 0: each A_ff^-1 of the fluid solve is that many V-cycle-preconditioned GMRES steps
    variant: str = "ldu"           # block factorisation: "ldu" (Alg. 2), "lower", "upper", "diag"


class Blocks:
    """Class sub-blocks of the monolithic matrix (offsets m|s_v|s_u|f_v|f_p|n)."""

    def __init__(self, A: sp.csr_matrix, offsets, dim: int):
        A = sp.csr_matrix(A)
        o = [int(v) for v in offsets]
        self.o, self.dim = o, dim
        self.m = slice(o[0], o[1])
        self.sv = slice(o[1], o[2])
        self.su = slice(o[2], o[3])
        self.fv = slice(o[3], o[4])
        self.p = slice(o[4], o[5])
        self.s = slice(o[1], o[3])
        self.f = slice(o[3], o[5])

        def blk(r, c):
            B = A[r, c].tocsr()
            B.sort_indices()
            return B
        self.M, self.C_ms = blk(self.m, self.m), blk(self.m, self.s)
        self.C_sm = blk(self.s, self.m)
        self.S = blk(self.s, self.s)
        self.A_vv, self.A_vu = blk(self.sv, self.sv), blk(self.sv, self.su)
        self.A_uv, self.A_uu = blk(self.su, self.sv), blk(self.su, self.su)
        self.C_sf = blk(self.s, self.f)
        self.C_fm, self.C_fs = blk(self.f, self.m), blk(self.f, self.s)
        self.F = blk(self.f, self.f)
        self.A_ff, self.B_vp = blk(self.fv, self.fv), blk(self.fv, self.p)
        self.B_pv, self.C_pp = blk(self.p, self.fv), blk(self.p, self.p)


def solid_schur(blocks: Blocks, c: float) -> sp.csr_matrix:
    """S_hat = A_vv + c A_vu (Alg. 3)."""
    S = (blocks.A_vv + c * blocks.A_vu).tocsr()
    S.sort_indices()
    return S


def pressure_schur(blocks: Blocks) -> sp.csr_matrix:
    """S_p = C_pp - B_pv diag(A_ff)^-1 B_vp."""
    dinv = 1.0 / blocks.A_ff.diagonal()
    S = (blocks.C_pp - blocks.B_pv @ sp.diags(dinv) @ blocks.B_vp).tocsr()
    S.sort_indices()
    return S


class _AMGInverse:
    def __init__(self, A, b, B, params: AMGParams, ncycles: int):
        self.A = A
        self.H = sa_setup(A, b, B, params)
        self.ncycles = ncycles

    def __call__(self, r):
        x = vcycle(self.H, r)
        for _ in range(1, self.ncycles):
            x = x + vcycle(self.H, r - self.A @ x)
        return x


class _ChebInverse:
    def __init__(self, A, degree, ratio, upper, power_iters):
        self.A = A
        self.dinv = point_dinv(A)
        self.lam = power_lambda(A, self.dinv, power_iters, 0)
        self.degree, self.ratio, self.upper = degree, ratio, upper

    def __call__(self, r):
        return chebyshev(self.A, self.dinv, r, None, self.lam, self.degree, self.ratio, self.upper, x_is_zero=True)


class _GMRESInverse:
    """x_k of k steps of GMRES on A x = r from x = 0, right-preconditioned by M
    (x_k minimises ||r - A x|| over x in M K_k(A M, r)); no stopping test."""

    def __init__(self, A, M, k: int):
        self.A, self.M, self.k = A, M, k

    def __call__(self, r):
        return fgmres(lambda v: self.A @ v, self.M, r, tol=0.0, restart=self.k, maxit=self.k).x


class _ExactInverse:
    def __init__(self, A):
        self.lu = spla.splu(sp.csc_matrix(A))

    def __call__(self, r):
        return self.lu.solve(r)


class BlockLDU:
    """P^-1 r of Alg. 2 with AMG sub-solves (or exact ones when exact=True)."""

    def __init__(self, A: sp.csr_matrix, offsets, dim: int, solid_coords=None,
                 params: PrecondParams | None = None, exact: bool = False):
        self.params = params = params or PrecondParams()
        self.B = B = Blocks(A, offsets, dim)
        self.S_hat = solid_schur(B, params.dt_theta)
        self.S_p = pressure_schur(B)
        d = dim
        if exact:
            self.M_inv = _ExactInverse(B.M)
            self.S_inv_exact = _ExactInverse(B.S)
            self.F_inv_exact = _ExactInverse(B.F)
            return
        self.S_inv_exact = self.F_inv_exact = None
        ap = params.amg
        self.M_inv = _AMGInverse(B.M, d, translations(B.M.shape[0] // d, d), ap, params.vcycles_mesh)
        ns = rigid_body_modes(solid_coords) if solid_coords is not None else \
            translations(self.S_hat.shape[0] // d, d)
        self.Shat_inv = _AMGInverse(self.S_hat, d, ns, ap, params.vcycles_solid)
        self.Ms_inv = _ChebInverse(B.A_uu, params.mass_degree, params.mass_ratio, ap.cheb_upper, ap.power_iters)
        # dt*theta on the s_u rows A_uv couples (the free rows), 0 on the fixed ones
        self.uv_weight = np.where(np.diff(sp.csr_matrix(B.A_uv).indptr) > 0, params.dt_theta, 0.0)
        self.Aff_inv = _AMGInverse(B.A_ff, d, translations(B.A_ff.shape[0] // d, d), ap, params.vcycles_fluid)
        if params.fluid_gmres_iters > 0:
            self.Aff_inv = _GMRESInverse(B.A_ff, self.Aff_inv, params.fluid_gmres_iters)
        self.Sp_inv = _AMGInverse(self.S_p, 1, np.ones((self.S_p.shape[0], 1)), ap, params.vcycles_pressure)

    # -------------------------------------------------------- sub-solves
    def S_inv(self, r_s):
        """Solid sub-solve, Alg. 3."""
        if self.S_inv_exact is not None:
            return self.S_inv_exact(r_s)
        B = self.B
        nv = B.A_vv.shape[0]
        r_v, r_u = r_s[:nv], r_s[nv:]
        y = self.Ms_inv(r_u)
        x_v = self.Shat_inv(r_v - B.A_vu @ y)
        x_u = y + self.uv_weight * x_v
        return np.concatenate([x_v, x_u])

    def F_inv(self, r_f):
        """Fluid sub-solve: pressure Schur complement elimination."""
        if self.F_inv_exact is not None:
            return self.F_inv_exact(r_f)
        B = self.B
        nv = B.A_ff.shape[0]
        r_v, r_p = r_f[:nv], r_f[nv:]
        y_v = self.Aff_inv(r_v)
        x_p = self.Sp_inv(r_p - B.B_pv @ y_v)
        x_v = self.Aff_inv(r_v - B.B_vp @ x_p)
        return np.concatenate([x_v, x_p])

    # -------------------------------------------------------- Alg. 2
    def __call__(self, r):
        B = self.B
        r_m, r_s, r_f = r[B.m], r[B.s], r[B.f]
        v = self.params.variant
        if v == "diag":                                    # D^-1
            return np.concatenate([self.M_inv(r_m), self.S_inv(r_s), self.F_inv(r_f)])
        if v == "upper":                                   # (D + U)^-1, backward substitution
            x_f = self.F_inv(r_f)
            x_s = self.S_inv(r_s - B.C_sf @ x_f)
            x_m = self.M_inv(r_m - B.C_ms @ x_s)
            return np.concatenate([x_m, x_s, x_f])
        x_m = self.M_inv(r_m)
        x_s = self.S_inv(r_s)
        x_f = self.F_inv(r_f - B.C_fm @ x_m - B.C_fs @ x_s)
        if v == "lower":                                   # (D + L)^-1: steps 1-3
            return np.concatenate([x_m, x_s, x_f])
        if v != "ldu":
            raise ValueError(f"unknown variant {v!r}")
        x_s = x_s - self.S_inv(B.C_sf @ x_f)
        x_m = x_m - self.M_inv(B.C_ms @ x_s)
        return np.concatenate([x_m, x_s, x_f])
