"""Smoothed-aggregation AMG (Vanek, Mandel & Brezina, Computing 56, 1996), the
sub-solver the paper applies to the mesh, solid and fluid blocks (Sec. 4.2-4.4,
which name Trilinos ML but fix none of its parameters).  Oracle copy: plain
numpy/scipy, FP64, test infrastructure only.

Set-up per level (the reading the CUDA path implements independently):
  1. strength: block Frobenius norms f_ij of the b x b node blocks, squares summed
     in row-major order; j != i is a strong neighbour of i when
     max(f_ij, f_ji) > 0 and max(f_ij, f_ji) >= theta * sqrt(f_ii * f_jj)
     (f_ji = 0 when that block is absent);
  2. aggregation: distance-2 maximal independent set of the strength graph
     (Bell, Dalton & Olson, SIAM J. Sci. Comput. 34, 2012) with node keys
     (state, priority, index), priorities from SplitMix64; roots seed
     aggregates, their neighbours join them, then every remaining node joins the
     aggregated neighbour of largest (priority, index).  Nodes without strong
     neighbours stay unaggregated;
  3. tentative prolongator: per aggregate, modified Gram-Schmidt on the
     near-nullspace rows of its nodes (columns whose remaining norm falls below
     drop_tol times their initial norm are dropped); Q fills P_tent, R is the
     coarse near-nullspace;
  4. lambda = |lambda_max(D^-1 A)| by power iteration (D = point diagonal);
     P = (I - omega D^-1 A) P_tent with omega = 4 / (3 lambda);
  5. R = P^T, A_c = R (A P).
Smoother: Chebyshev iteration (Saad, Iterative Methods, 2nd ed., Alg. 12.1) on
D^-1 A over [lambda / cheb_ratio, cheb_upper * lambda].  Coarsest level: dense
solve (all-zero rows replaced by identity rows).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .splitmix import node_priority, unit_uniform

IDX_BITS = 27          # node index bits in the aggregation key (n < 2^27)
STATE_SHIFT = 59       # key = state << 59 | priority << 27 | index


@dataclass
class AMGParams:
    theta: float = 0.08
    coarse_max: int = 1500       # stop coarsening at <= this many scalar rows
    max_levels: int = 10
    cheb_degree: int = 4
    cheb_ratio: float = 30.0
    cheb_upper: float = 1.3
    power_iters: int = 15
    drop_tol: float = 1e-10
    presmooth: int = 1
    postsmooth: int = 1
    cheb_degree_coarse: int = 2  # Chebyshev degree on levels >= 1 (0: cheb_degree everywhere)

    def degree(self, level: int) -> int:
        return self.cheb_degree_coarse if level > 0 and self.cheb_degree_coarse > 0 else self.cheb_degree


# ------------------------------------------------------------------ set-up
def block_frobenius(data: np.ndarray) -> np.ndarray:
    """Frobenius norm of each (b x b) block, squares added in row-major order."""
    nb, br, bc = data.shape
    s = data[:, 0, 0] * data[:, 0, 0]
    for i in range(br):
        for j in range(bc):
            if i == 0 and j == 0:
                continue
            s = s + data[:, i, j] * data[:, i, j]
    return np.sqrt(s)


def strength_graph(A: sp.csr_matrix, b: int, theta: float) -> sp.csr_matrix:
    """Symmetric strong-connection graph between the nodes (b x b blocks) of A."""
    nb = A.shape[0] // b
    Ab = sp.bsr_matrix(A, blocksize=(b, b))
    Ab.sort_indices()
    f = block_frobenius(Ab.data)
    N = sp.csr_matrix((f, Ab.indices, Ab.indptr), shape=(nb, nb))
    diag = N.diagonal()
    S = N.maximum(N.T.tocsr()).tocoo()
    i, j, v = S.row, S.col, S.data
    thr = theta * np.sqrt(diag[i] * diag[j])
    keep = (i != j) & (v > 0.0) & (v >= thr)
    G = sp.csr_matrix((np.ones(int(keep.sum())), (i[keep], j[keep])), shape=(nb, nb))
    G.sort_indices()
    return G


def _row_max(G: sp.csr_matrix, vals: np.ndarray) -> np.ndarray:
    """max over each row's entries of vals[col] (rows must be non-empty)."""
    return np.maximum.reduceat(vals[G.indices], G.indptr[:-1])


def aggregate(G: sp.csr_matrix, level: int):
    """Distance-2 MIS aggregation.  Returns (agg id per node or -1, #aggregates)."""
    n = G.shape[0]
    if n >= (1 << IDX_BITS):
        raise ValueError("too many nodes for the aggregation key")
    deg = np.diff(G.indptr)
    isolated = deg == 0
    Gs = (G + sp.identity(n, format="csr")).tocsr()
    Gs.sort_indices()
    idx = np.arange(n, dtype=np.int64)
    base = (node_priority(n, level) << IDX_BITS) | idx
    state = np.where(isolated, 0, 1).astype(np.int64)       # 0 out, 1 undecided, 2 in
    while np.any(state == 1):
        key = (state << STATE_SHIFT) | base
        t2 = _row_max(Gs, _row_max(Gs, key))
        und = state == 1
        new_in = und & (t2 == key)
        new_out = und & ~new_in & ((t2 >> STATE_SHIFT) == 2)
        state[new_in] = 2
        state[new_out] = 0
    roots = state == 2
    agg = np.full(n, -1, np.int64)
    nagg = int(roots.sum())
    agg[roots] = np.arange(nagg)
    rows = np.repeat(idx, deg)
    cols = G.indices.astype(np.int64)
    m = roots[cols] & ~roots[rows]
    agg[rows[m]] = agg[cols[m]]
    first = agg >= 0
    todo = (~first) & (~isolated)
    if np.any(todo):
        cand = np.where(first, base, -1)
        best = _row_max(Gs, cand)
        if np.any(best[todo] < 0):
            raise RuntimeError("aggregation left a node without an aggregated neighbour")
        agg[todo] = agg[best[todo] & ((1 << IDX_BITS) - 1)]
    return agg, nagg


def mgs(Bj: np.ndarray, drop_tol: float):
    """Modified Gram-Schmidt thin QR with positive diagonal; dropped columns give
    zero columns of Q and zero rows of R."""
    m, k = Bj.shape
    Q = Bj.astype(np.float64).copy()
    R = np.zeros((k, k))
    for c in range(k):
        q = Q[:, c]
        orig = np.sqrt(np.dot(q, q))
        for j in range(c):
            rjc = np.dot(Q[:, j], q)
            R[j, c] = rjc
            q = q - rjc * Q[:, j]
        nrm = np.sqrt(np.dot(q, q))
        if orig == 0.0 or nrm <= drop_tol * orig:
            Q[:, c] = 0.0
            R[c, c] = 0.0
        else:
            Q[:, c] = q / nrm
            R[c, c] = nrm
    return Q, R


def tentative_prolongator(agg: np.ndarray, nagg: int, B: np.ndarray, b: int, drop_tol: float):
    """P_tent (BSR, b x k blocks) and coarse near-nullspace B_c (nagg*k x k)."""
    n = agg.shape[0]
    k = B.shape[1]
    Bn = B.reshape(n, b, k)
    order = np.argsort(agg, kind="stable")
    order = order[agg[order] >= 0]
    starts = np.searchsorted(agg[order], np.arange(nagg + 1))
    blocks = np.zeros((n, b, k))
    Bc = np.zeros((nagg, k, k))
    for J in range(nagg):
        members = order[starts[J]:starts[J + 1]]
        Q, R = mgs(Bn[members].reshape(-1, k), drop_tol)
        blocks[members] = Q.reshape(len(members), b, k)
        Bc[J] = R
    has = agg >= 0
    indptr = np.concatenate([[0], np.cumsum(has)]).astype(np.int64)
    P = sp.bsr_matrix((blocks[has], agg[has], indptr), shape=(n * b, nagg * k))
    return P, Bc.reshape(nagg * k, k)


def point_dinv(A: sp.csr_matrix) -> np.ndarray:
    d = A.diagonal()
    out = np.zeros_like(d)
    nz = d != 0.0
    out[nz] = 1.0 / d[nz]
    return out


def power_lambda(A: sp.csr_matrix, dinv: np.ndarray, iters: int, level: int) -> float:
    """|lambda_max(D^-1 A)| estimate: power iteration from x_i = 1 + u_i (SplitMix64
    stream 256 + level)."""
    if A.shape[0] == 0:
        return 0.0            # an empty operator (a block with no DOFs) has no spectrum
    x = 1.0 + unit_uniform(A.shape[0], 256 + level)
    lam = 0.0
    for _ in range(iters):
        y = dinv * (A @ x)
        ny = np.sqrt(np.dot(y, y))
        nx = np.sqrt(np.dot(x, x))
        lam = ny / nx
        if ny == 0.0:
            break
        x = y / ny
    return lam


@dataclass
class Level:
    A: sp.csr_matrix
    b: int
    dinv: np.ndarray
    lam: float
    P: sp.csr_matrix | None = None
    R: sp.csr_matrix | None = None
    agg: np.ndarray | None = None
    nagg: int = 0


@dataclass
class Hierarchy:
    levels: list
    coarse_inv: np.ndarray
    params: AMGParams = field(default_factory=AMGParams)

    def operator_complexity(self) -> float:
        return sum(L.A.nnz for L in self.levels) / self.levels[0].A.nnz


def coarse_dense_inverse(A: sp.csr_matrix) -> np.ndarray:
    D = A.toarray()
    zero = ~np.any(D != 0.0, axis=1)
    D[zero, zero] = 1.0
    return sla.inv(D)


def sa_setup(A: sp.csr_matrix, b: int, B: np.ndarray, params: AMGParams | None = None) -> Hierarchy:
    """Build the smoothed-aggregation hierarchy of A (block size b, near-nullspace B)."""
    params = params or AMGParams()
    A = sp.csr_matrix(A)
    A.sort_indices()
    levels = []
    lvl = 0
    while True:
        dinv = point_dinv(A)
        lam = power_lambda(A, dinv, params.power_iters, lvl)
        L = Level(A=A, b=b, dinv=dinv, lam=lam)
        levels.append(L)
        if A.shape[0] <= params.coarse_max or lvl + 1 >= params.max_levels:
            break
        G = strength_graph(A, b, params.theta)
        agg, nagg = aggregate(G, lvl)
        k = B.shape[1]
        if nagg == 0 or nagg * k >= A.shape[0]:
            break
        Pt, Bc = tentative_prolongator(agg, nagg, B, b, params.drop_tol)
        Pt = Pt.tocsr()
        omega = 4.0 / (3.0 * lam)
        AP = (A @ Pt).tocsr()
        P = (Pt - sp.diags(omega * dinv) @ AP).tocsr()
        R = P.T.tocsr()
        Ac = (R @ (A @ P)).tocsr()
        Ac.sort_indices()
        L.P, L.R, L.agg, L.nagg = P, R, agg, nagg
        A, B, b = Ac, Bc, k
        lvl += 1
    return Hierarchy(levels=levels, coarse_inv=coarse_dense_inverse(levels[-1].A), params=params)


# ------------------------------------------------------------------ apply
def chebyshev(A, dinv, b, x, lam, degree, ratio, upper, x_is_zero=False):
    """Chebyshev iteration on D^-1 A x = D^-1 b over [lam/ratio, upper*lam]
    (Saad Alg. 12.1, residual recomputed every step)."""
    beta = upper * lam
    alpha = lam / ratio
    theta = 0.5 * (beta + alpha)
    delta = 0.5 * (beta - alpha)
    sigma = theta / delta
    rho = 1.0 / sigma
    r = dinv * b if x_is_zero else dinv * (b - A @ x)
    d = r / theta
    x = d.copy() if x_is_zero else x + d
    for _ in range(1, degree):
        r = dinv * (b - A @ x)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = (rho_new * rho) * d + (2.0 * rho_new / delta) * r
        x = x + d
        rho = rho_new
    return x


def vcycle(H: Hierarchy, b: np.ndarray, lvl: int = 0) -> np.ndarray:
    """One V-cycle for A_lvl x = b from x = 0."""
    p = H.params
    L = H.levels[lvl]
    if lvl == len(H.levels) - 1:
        return H.coarse_inv @ b
    x = None
    for s in range(p.presmooth):
        x = chebyshev(L.A, L.dinv, b, x, L.lam, p.degree(lvl), p.cheb_ratio, p.cheb_upper, x_is_zero=(s == 0))
    r = b - L.A @ x
    xc = vcycle(H, L.R @ r, lvl + 1)
    x = x + L.P @ xc
    for _ in range(p.postsmooth):
        x = chebyshev(L.A, L.dinv, b, x, L.lam, p.degree(lvl), p.cheb_ratio, p.cheb_upper)
    return x


# ------------------------------------------------------------------ near-nullspaces
def translations(n_nodes: int, b: int) -> np.ndarray:
    """b rigid translations of a b-component vector field (node-major)."""
    return np.tile(np.eye(b), (n_nodes, 1))


def rigid_body_modes(coords: np.ndarray) -> np.ndarray:
    """Translations and infinitesimal rotations about the origin: 3 modes in 2D,
    6 in 3D (node-major, component-minor)."""
    n, d = coords.shape
    x = coords
    if d == 2:
        B = np.zeros((n, 2, 3))
        B[:, 0, 0] = 1.0
        B[:, 1, 1] = 1.0
        B[:, 0, 2] = -x[:, 1]
        B[:, 1, 2] = x[:, 0]
        return B.reshape(2 * n, 3)
    B = np.zeros((n, 3, 6))
    for c in range(3):
        B[:, c, c] = 1.0
    # rotations about z, x, y: (-y, x, 0), (0, -z, y), (z, 0, -x)
    B[:, 0, 3], B[:, 1, 3] = -x[:, 1], x[:, 0]
    B[:, 1, 4], B[:, 2, 4] = -x[:, 2], x[:, 1]
    B[:, 2, 5], B[:, 0, 5] = -x[:, 0], x[:, 2]
    return B.reshape(3 * n, 6)
