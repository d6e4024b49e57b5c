"""Pins of two oracle set-up formulas that the solve tests only see through their
effect on convergence:

* the pressure Schur approximation S_p = C_pp - B_pv diag(A_ff)^-1 B_vp of the
  fluid sub-solve (Sec. 4.4, SIMPLE-type reading), by a 2-velocity-node /
  2-pressure-node example whose S_p is worked out by hand below, and by the
  exactness of the fluid Schur elimination when A_ff is replaced by its
  diagonal: with exact inverses of D = diag(A_ff) and of S_p, F_inv solves
  F_D = [[D, B_vp], [B_pv, C_pp]] exactly (block LU of F_D);
* the strength-of-connection rule of the SA-AMG set-up (block Frobenius norms,
  symmetrised by the larger of f_ij and f_ji, strong iff >= theta sqrt(f_ii f_jj),
  theta = 0.08), by hand-worked scalar and 2 x 2-block examples.

Each example is built so that a plausible slip gives another answer: a sign slip
or row sums instead of the diagonal in S_p, B_vp and B_pv swapped, min instead
of max, only the own row's entry, > instead of >=, the largest entry or the
entry sum instead of the Frobenius norm."""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

import fsigen
import oracle
from oracle.amg import strength_graph
from oracle.precond import Blocks, pressure_schur


def _fluid_only_system(A_ff, B_vp, B_pv, C_pp):
    """Monolithic matrix with empty m / s classes: offsets 0|0|0|0|n_v|n_v+n_p."""
    nv, npr = A_ff.shape[0], C_pp.shape[0]
    A = np.block([[A_ff, B_vp], [B_pv, C_pp]])
    return sp.csr_matrix(A), [0, 0, 0, 0, nv, nv + npr]


def test_pressure_schur_hand_example():
    # two velocity nodes (4 DOFs, d = 2), two pressure nodes
    A_ff = np.array([[2.0, 1.0, 0.0, 0.0],
                     [0.0, 4.0, 0.0, 0.0],
                     [0.0, 0.0, 5.0, 1.0],
                     [1.0, 0.0, 0.0, 10.0]])
    B_vp = np.array([[1.0, 0.0], [-2.0, 1.0], [3.0, 0.0], [0.5, 2.0]])
    B_pv = np.array([[2.0, 1.0, -1.0, 4.0], [0.0, 3.0, 0.0, 1.0]])
    C_pp = np.array([[0.25, 0.0], [0.0, -0.5]])
    A, off = _fluid_only_system(A_ff, B_vp, B_pv, C_pp)
    S = pressure_schur(Blocks(A, off, 2)).toarray()
    # By hand: diag(A_ff)^-1 = diag(1/2, 1/4, 1/5, 1/10);
    #   D^-1 B_vp = [[0.5, 0], [-0.5, 0.25], [0.6, 0], [0.05, 0.2]]
    #   B_pv D^-1 B_vp = [[2*0.5 - 0.5 - 0.6 + 4*0.05, 0.25 + 4*0.2],
    #                     [3*(-0.5) + 0.05,           3*0.25 + 0.2]] = [[0.1, 1.05], [-1.45, 0.95]]
    #   S_p = C_pp - that = [[0.15, -1.05], [1.45, -1.45]]
    expect = np.array([[0.15, -1.05], [1.45, -1.45]])
    assert np.allclose(S, expect, rtol=0, atol=1e-14)
    # what the slips would give (none of them is the expected matrix)
    assert not np.allclose(np.array([[0.35, 1.05], [-1.45, 0.45]]), expect)    # sign slip: C_pp + ...
    assert not np.allclose(np.array([[0.15, 1.45], [-1.05, -1.45]]), expect)   # B_vp^T D^-1 B_pv^T


def test_pressure_schur_makes_the_diagonal_fluid_elimination_exact():
    s = fsigen.make_system(fsigen.CONFIGS["2d_tiny"].with_(name="o2", n=(8, 8)))
    pre = oracle.BlockLDU(s.scipy(), s.offsets, 2, s.solid_coords, oracle.PrecondParams(mass_ratio=8.0))
    B = pre.B
    d = B.A_ff.diagonal()
    assert np.all(d != 0.0)
    S_p = pressure_schur(B).toarray()
    lu = sla.lu_factor(S_p)
    pre.Aff_inv = lambda r: r / d                  # exact inverse of D = diag(A_ff)
    pre.Sp_inv = lambda r: sla.lu_solve(lu, r)     # exact inverse of S_p
    F_D = np.block([[np.diag(d), B.B_vp.toarray()], [B.B_pv.toarray(), B.C_pp.toarray()]])
    r = np.random.default_rng(7).standard_normal(F_D.shape[0])
    x = pre.F_inv(r)
    xd = np.linalg.solve(F_D, r)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    assert np.linalg.norm(F_D @ x - r) <= 1e-10 * np.linalg.norm(r) * np.abs(F_D).max()


def _edges(G):
    G = G.tocoo()
    return {(int(i), int(j)) for i, j in zip(G.row, G.col)}


def test_strength_graph_scalar_hand_example():
    A = np.array([[4.0, -1.0, 0.1, 0.0],
                  [-1.0, 4.0, 0.0, -0.2],
                  [0.0, 0.5, 1.0, 0.08],
                  [0.0, 0.2, 0.0, 1.0]])
    G = strength_graph(sp.csr_matrix(A), 1, 0.08)
    # By hand (f = |a|, thr_ij = 0.08 sqrt(f_ii f_jj)):
    #   0-1: max(1, 1) = 1      >= 0.08*4 = 0.32   strong
    #   0-2: max(0.1, 0) = 0.1  <  0.08*2 = 0.16   weak   (one-sided entry)
    #   1-2: max(0, 0.5) = 0.5  >= 0.16            strong (only row 2 holds the entry)
    #   1-3: max(0.2, 0.2)      >= 0.16            strong
    #   2-3: max(0.08, 0)       >= 0.08*1 = 0.08   strong (equality counts)
    #   0-3: no entries                            weak
    strong = {(0, 1), (1, 2), (1, 3), (2, 3)}
    assert _edges(G) == strong | {(j, i) for i, j in strong}
    assert np.all(G.data == 1.0)


def test_strength_graph_block_hand_example():
    # three nodes with 2 x 2 blocks
    blocks = {
        (0, 0): [[3.0, 0.0], [0.0, 4.0]],      # f = 5
        (1, 1): [[0.6, 0.0], [0.0, 0.8]],      # f = 1
        (2, 2): [[1.0, 0.0], [0.0, 0.0]],      # f = 1
        (0, 1): [[0.12, 0.12], [0.12, 0.0]],   # f = sqrt(3*0.0144) = 0.2078 >= 0.08 sqrt(5) = 0.1789
        (0, 2): [[0.1, 0.1], [0.0, 0.0]],      # f = sqrt(0.02) = 0.1414 < 0.1789 (entry sum 0.2 would pass)
        (1, 2): [[0.05, 0.0], [0.0, 0.0]],     # f = 0.05
        (2, 1): [[0.0, 0.09], [0.0, 0.0]],     # f = 0.09 >= 0.08 sqrt(1*1) = 0.08
    }
    A = np.zeros((6, 6))
    for (i, j), b in blocks.items():
        A[2 * i:2 * i + 2, 2 * j:2 * j + 2] = b
    G = strength_graph(sp.csr_matrix(A), 2, 0.08)
    # 0-1 strong by the Frobenius norm (the largest entry 0.12 would fail), 0-2 weak,
    # 1-2 strong through the larger of the two directions
    strong = {(0, 1), (1, 2)}
    assert _edges(G) == strong | {(j, i) for i, j in strong}
