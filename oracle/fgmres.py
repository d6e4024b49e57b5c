"""Right-preconditioned flexible GMRES (Saad, Iterative Methods for Sparse Linear
Systems, 2nd ed., Alg. 9.6) with Givens rotations for the Hessenberg
least-squares problem.  The Arnoldi step orthogonalises by classical
Gram-Schmidt applied twice (Giraud, Langou & Rozloznik, Comput. Math. Appl. 50,
2005: "twice is enough"): on these badly scaled Jacobians (condition numbers
near 1e14) single-pass modified Gram-Schmidt loses orthogonality and stalls.  The paper solves each
Newton step's system A_h dU = F_h with GMRES preconditioned by Alg. 2 (Sec. 4,
Sec. 6 solver settings); the stopping rule here is the relative residual
||b - A x|| / ||b|| <= tol, checked on the Givens estimate and confirmed on the
true residual before returning.  Oracle copy: test infrastructure only.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class FGMRESResult:
    x: np.ndarray
    iters: int
    cycles: int
    converged: bool
    true_relres: float
    history: list = field(default_factory=list)   # |g_{j+1}| / ||b|| per iteration
    breakdown: bool = False
    cycle_starts: list = field(default_factory=list)   # index into history where each cycle starts
    accepted: int = 0                                  # learned-stage corrections taken


def fgmres(A, M, b, tol=1e-8, restart=100, maxit=1000, x0=None, correct=None, accept=1.0) -> FGMRESResult:
    """Solve A x = b; A(x) and M(r) are callables (matrix-vector and P^-1).

    correct(r') -> c, if given, is the learned stage: with q = A z_j and
    r' = v_j - q, the correction c is taken (z_j += c, w = q + A c) only when
    ||r' - A c|| < accept * ||r'||; otherwise w = q as without the stage."""
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.sqrt(np.dot(b, b))
    if bnorm == 0.0:
        return FGMRESResult(np.zeros(n), 0, 0, True, 0.0)
    hist = []
    starts = []
    total = 0
    cycles = 0
    breakdown = False
    accepted = 0
    while True:
        r = b - A(x)
        beta = np.sqrt(np.dot(r, r))
        if beta / bnorm <= tol:
            return FGMRESResult(x, total, cycles, True, beta / bnorm, hist, breakdown, starts, accepted)
        if total >= maxit:
            return FGMRESResult(x, total, cycles, False, beta / bnorm, hist, breakdown, starts, accepted)
        starts.append(len(hist))
        m = restart
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_end = 0
        for j in range(m):
            Z[j] = M(V[j])
            w = A(Z[j])
            if correct is not None:
                rp = V[j] - w
                c = correct(rp)
                t = A(c)
                d = rp - t
                if np.dot(d, d) < accept * accept * np.dot(rp, rp):
                    Z[j] = Z[j] + c
                    w = w + t
                    accepted += 1
            wnorm0 = np.sqrt(np.dot(w, w))
            for _ in range(2):                      # classical Gram-Schmidt, twice
                h = V[:j + 1] @ w
                w = w - V[:j + 1].T @ h
                H[:j + 1, j] += h
            H[j + 1, j] = np.sqrt(np.dot(w, w))
            # apply the previous rotations to column j, then form the new one
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            hj1 = H[j + 1, j]
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            j_end = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if hj1 <= 1e-14 * wnorm0:
                breakdown = True
                break
            V[j + 1] = w / hj1
            if abs(g[j + 1]) / bnorm <= tol or total >= maxit:
                break
        # x = x0 + Z y,  H y = g  (upper triangular)
        k = j_end
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        x = x + Z[:k].T @ y
        cycles += 1
        if breakdown:
            r = b - A(x)
            rel = np.sqrt(np.dot(r, r)) / bnorm
            return FGMRESResult(x, total, cycles, rel <= tol, rel, hist, breakdown, starts, accepted)
