"""Pins of the oracle's Alg. 2 preconditioner and FGMRES on tiny seeded FSI
systems: dense LU brute force, the exact-sub-solve identity
P = (D + L) D^-1 (D + U), the <= 3-iteration bound for exact block-triangular
preconditioning, exact LDU = 1 iteration, monotone residuals, and the Givens
least-squares estimate equal to the true residual and to lstsq."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import fsigen
import oracle
from oracle.fgmres import fgmres


def tiny(dim):
    if dim == 2:
        return fsigen.make_system(fsigen.CONFIGS["2d_tiny"].with_(name="o2", n=(8, 8)))
    return fsigen.make_system(fsigen.CONFIGS["3d"].with_(name="o3", n=(4, 2, 4)))


def params(dim):
    return oracle.PrecondParams(mass_ratio=8.0 if dim == 2 else 20.0)


@pytest.mark.parametrize("dim", [2, 3])
def test_fgmres_alg2_matches_dense_lu(dim):
    s = tiny(dim)
    A = s.scipy()
    xd = sla.solve(A.toarray(), s.rhs)
    # dense LU recovers the manufactured solution (condition number ~1e14, b = A x*)
    assert np.linalg.norm(xd - s.x_exact) / np.linalg.norm(s.x_exact) <= 1e-7
    o = oracle.OracleSolver.from_system(s, params(dim))
    r = o.solve(s.rhs, tol=1e-8)
    assert r.converged and r.true_relres <= 1e-8
    kappa_bound = np.linalg.cond(A.toarray(), 1)
    err = np.linalg.norm(r.x - xd) / np.linalg.norm(xd)
    assert err <= kappa_bound * 1e-8
    # tightening the tolerance drives FGMRES onto the direct solution
    errs = []
    for tol in (1e-8, 1e-10, 1e-12):
        rt = o.solve(s.rhs, tol=tol, restart=200)
        assert rt.converged
        errs.append(np.linalg.norm(rt.x - xd) / np.linalg.norm(xd))
    assert errs[0] > errs[1] > errs[2] and errs[2] <= 1e-4
    # within a cycle the residual estimate never increases (nested Krylov spaces)
    bounds = list(r.cycle_starts) + [len(r.history)]
    for a, b in zip(bounds[:-1], bounds[1:]):
        h = np.array(r.history[a:b])
        assert np.all(np.diff(h) <= 1e-14)


def _dense_blocks(s):
    A = s.scipy().toarray()
    o = s.offsets
    I = [slice(o[0], o[1]), slice(o[1], o[3]), slice(o[3], o[5])]
    return A, I


def test_exact_alg2_is_block_symmetric_gauss_seidel():
    s = tiny(2)
    A, I = _dense_blocks(s)
    D = np.zeros_like(A)
    L = np.zeros_like(A)
    U = np.zeros_like(A)
    for a in range(3):
        for b in range(3):
            blk = A[I[a], I[b]]
            if a == b:
                D[I[a], I[b]] = blk
            elif a > b and not (a == 1 and b == 0):     # C_sm dropped
                L[I[a], I[b]] = blk
            elif a < b:
                U[I[a], I[b]] = blk
    P = (D + L) @ np.linalg.solve(D, D + U)
    pre = oracle.BlockLDU(s.scipy(), s.offsets, 2, exact=True)
    r = np.random.default_rng(5).standard_normal(A.shape[0])
    assert np.allclose(pre(r), np.linalg.solve(P, r), rtol=1e-9, atol=1e-9 * np.abs(np.linalg.solve(P, r)).max())


def test_exact_block_triangular_converges_in_three_iterations():
    """T = L D = [[M,0,0],[C_sm,S1,0],[C_fm,C~_fs,X]] of the exact LDU (Sec. 4.1) with
    the true Schur complements: T^-1 A = U is unit block upper triangular, so
    (T^-1 A - I)^3 = 0 and GMRES stops within 3 iterations.  The system is first
    equilibrated by diagonal row and column scalings (which keep the block
    structure and the theorem) so that rounding stays far below the tolerance."""
    s = tiny(2)
    A, I = _dense_blocks(s)
    rs = 1.0 / np.abs(A).max(axis=1)
    A = rs[:, None] * A
    cs = 1.0 / np.abs(A).max(axis=0)
    A = A * cs[None, :]
    rhs = rs * s.rhs
    M, Cms = A[I[0], I[0]], A[I[0], I[1]]
    Csm, S, Csf = A[I[1], I[0]], A[I[1], I[1]], A[I[1], I[2]]
    Cfm, Cfs, F = A[I[2], I[0]], A[I[2], I[1]], A[I[2], I[2]]
    S1 = S - Csm @ np.linalg.solve(M, Cms)
    Cfs_t = Cfs - Cfm @ np.linalg.solve(M, Cms)
    X = F - Cfs_t @ np.linalg.solve(S1, Csf)
    T = np.zeros_like(A)
    T[I[0], I[0]] = M
    T[I[1], I[0]], T[I[1], I[1]] = Csm, S1
    T[I[2], I[0]], T[I[2], I[1]], T[I[2], I[2]] = Cfm, Cfs_t, X
    lu = sla.lu_factor(T)
    res = fgmres(lambda v: A @ v, lambda r: sla.lu_solve(lu, r), rhs, tol=1e-10, restart=20, maxit=20)
    assert res.converged and res.iters <= 3
    # full LDU with those factors reproduces A exactly: one iteration
    Lf = np.eye(A.shape[0])
    Lf[I[1], I[0]] = Csm @ np.linalg.inv(M)
    Lf[I[2], I[0]] = Cfm @ np.linalg.inv(M)
    Lf[I[2], I[1]] = Cfs_t @ np.linalg.inv(S1)
    Df = np.zeros_like(A)
    Df[I[0], I[0]], Df[I[1], I[1]], Df[I[2], I[2]] = M, S1, X
    Uf = np.eye(A.shape[0])
    Uf[I[0], I[1]] = np.linalg.solve(M, Cms)
    Uf[I[1], I[2]] = np.linalg.solve(S1, Csf)
    P = Lf @ Df @ Uf
    assert np.allclose(P, A, atol=1e-8 * np.abs(A).max())
    lu = sla.lu_factor(P)
    res = fgmres(lambda v: A @ v, lambda r: sla.lu_solve(lu, r), rhs, tol=1e-10, restart=20, maxit=20)
    assert res.converged and res.iters == 1


def test_solid_schur_alg3_with_exact_inverses_is_exact():
    s = tiny(2)
    pre = oracle.BlockLDU(s.scipy(), s.offsets, 2)
    B = pre.B
    from oracle.precond import _ExactInverse
    pre.Shat_inv = _ExactInverse(pre.S_hat)
    pre.Ms_inv = _ExactInverse(B.A_uu)
    r = np.random.default_rng(2).standard_normal(B.S.shape[0])
    x = pre.S_inv(r)
    x_direct = np.linalg.solve(B.S.toarray(), r)
    # an algebra slip shows as an O(1) difference; rounding (cond(S) ~ 1e9) stays << 1e-6
    assert np.linalg.norm(x - x_direct) <= 1e-6 * np.linalg.norm(x_direct)


@pytest.mark.parametrize("dim", [2, 3])
def test_solid_velocity_coupling_is_minus_dt_theta_mass(dim):
    """Alg. 3 applies one mass solve for both of its steps, which rests on
    A_uv = -dt*theta*A_uu on every free s_u row (the displacement equation
    (u - u_old) - dt*theta*v = 0 tested with the same Q2 basis) and on A_uv
    having no entries on fixed rows."""
    s = tiny(dim)
    pre = oracle.BlockLDU(s.scipy(), s.offsets, dim)
    B = pre.B
    c = pre.params.dt_theta
    fixed_u = s.fixed[B.su]
    D = (B.A_uv + c * B.A_uu).tocsr()
    assert abs(D[~fixed_u]).max() <= 1e-12 * abs(B.A_uu[~fixed_u]).max()
    assert B.A_uv.tocsr()[fixed_u].nnz == 0
    assert np.array_equal(pre.uv_weight, np.where(fixed_u, 0.0, c))


def test_fluid_schur_elimination_with_exact_schur_is_exact():
    s = tiny(2)
    pre = oracle.BlockLDU(s.scipy(), s.offsets, 2)
    B = pre.B
    from oracle.precond import _ExactInverse
    Aff = B.A_ff.toarray()
    Sp_exact = B.C_pp.toarray() - B.B_pv.toarray() @ np.linalg.solve(Aff, B.B_vp.toarray())
    pre.Aff_inv = _ExactInverse(B.A_ff)
    pre.Sp_inv = lambda r: np.linalg.solve(Sp_exact, r)
    r = np.random.default_rng(4).standard_normal(B.F.shape[0])
    x = pre.F_inv(r)
    x_direct = np.linalg.solve(B.F.toarray(), r)
    assert np.linalg.norm(x - x_direct) <= 1e-6 * np.linalg.norm(x_direct)


def test_givens_estimate_equals_true_residual_and_lstsq():
    s = tiny(2)
    A = s.scipy()
    pre = oracle.BlockLDU(A, s.offsets, 2, params=params(2))
    Zs = []
    rec = lambda r: (Zs.append(pre(r)), Zs[-1])[1]
    k = 3          # residual still far above the rounding floor of this ill-conditioned system
    res = fgmres(lambda v: A @ v, rec, s.rhs, tol=1e-30, restart=k, maxit=k)
    est = res.history[-1] * np.linalg.norm(s.rhs)
    true = np.linalg.norm(s.rhs - A @ res.x)
    assert est == pytest.approx(true, rel=1e-6)
    Z = np.column_stack(Zs)
    y, *_ = np.linalg.lstsq((A @ Z), s.rhs, rcond=None)
    assert np.linalg.norm(s.rhs - A @ (Z @ y)) == pytest.approx(true, rel=1e-6)


def test_large_amplitude_state_makes_the_solid_block_indefinite():
    """Why the 1024x512 case runs at amplitude 1e-2: at 5e-2 the seed-0 state
    compresses the solid so far that the St. Venant-Kirchhoff tangent, and with it
    S_hat = A_vv + dt A_vu (Alg. 3), is indefinite; the Chebyshev/AMG sub-solve
    cannot handle that.  At 1e-2 D^-1 S_hat keeps a positive real spectrum."""
    import scipy.sparse.linalg as spla
    from oracle.amg import point_dinv
    lo = {}
    for amp in (1e-2, 5e-2):
        s = fsigen.make_system(fsigen.CONFIGS["2d_tiny"].with_(name="amp", n=(32, 16), amplitude=amp))
        B = oracle.Blocks(s.scipy(), s.offsets, 2)
        S = oracle.solid_schur(B, 0.01)
        DS = sp.diags(point_dinv(S)) @ S
        ev = spla.eigs(DS, k=4, which="SR", return_eigenvectors=False)
        lo[amp] = float(np.min(ev.real))
    assert lo[1e-2] > 0.0
    assert lo[5e-2] < -0.5


def test_inner_gmres_returns_the_krylov_minimiser():
    """The fluid solve's inner GMRES (Sec. 4.4) against what k GMRES steps must
    return: with k = n the exact solution; after one step the minimal-residual
    multiple alpha M r; after k steps the minimiser of ||r - A x|| over
    x in M K_k(A M, r), computed here by least squares on an explicit basis."""
    from oracle.precond import _GMRESInverse
    rng = np.random.default_rng(11)
    n = 12
    A = 4.0 * np.eye(n) + rng.standard_normal((n, n))
    Mm = np.diag(1.0 / np.diag(A)) + 0.01 * rng.standard_normal((n, n))
    M = lambda v: Mm @ v
    r = rng.standard_normal(n)
    x = _GMRESInverse(A, M, n)(r)
    assert np.linalg.norm(A @ x - r) <= 1e-10 * np.linalg.norm(r)
    q = A @ (Mm @ r)
    alpha = (q @ r) / (q @ q)
    np.testing.assert_allclose(_GMRESInverse(A, M, 1)(r), alpha * (Mm @ r), rtol=1e-12, atol=1e-14)
    K = [r]
    for _ in range(3):
        K.append(A @ (Mm @ K[-1]))
    Q, _ = np.linalg.qr(np.column_stack(K))
    P = Mm @ Q
    c, *_ = np.linalg.lstsq(A @ P, r, rcond=None)
    x4 = _GMRESInverse(A, M, 4)(r)
    assert np.linalg.norm(x4 - P @ c) <= 1e-10 * np.linalg.norm(P @ c)


@pytest.mark.parametrize("dim", [2, 3])
def test_fluid_inner_gmres_improves_the_velocity_solve(dim):
    """k inner GMRES steps never leave a larger A_ff residual than the plain
    V-cycle (x = M r lies in the space they minimise over), and the outer solve
    still reaches the tolerance."""
    # 16x16 in 2D: A_ff needs more than one AMG level, so the V-cycle is not exact
    s = fsigen.make_system(fsigen.CONFIGS["2d_tiny"]) if dim == 2 else tiny(3)
    mr = 8.0 if dim == 2 else 20.0
    amg = oracle.AMGParams(coarse_max=500)     # keeps A_ff multi-level on these small meshes
    base = oracle.BlockLDU(s.scipy(), s.offsets, dim, params=oracle.PrecondParams(mass_ratio=mr, amg=amg))
    g4 = oracle.BlockLDU(s.scipy(), s.offsets, dim,
                         params=oracle.PrecondParams(mass_ratio=mr, fluid_gmres_iters=4, amg=amg))
    A_ff = base.B.A_ff
    r = np.random.default_rng(6).standard_normal(A_ff.shape[0])
    res = lambda x: np.linalg.norm(r - A_ff @ x)
    assert len(base.Aff_inv.H.levels) > 1
    r0 = res(base.Aff_inv(r))
    assert r0 > 1e-6 * np.linalg.norm(r)
    assert res(g4.Aff_inv(r)) <= r0 * (1 + 1e-12)
    o = oracle.OracleSolver.from_system(s, oracle.PrecondParams(mass_ratio=mr, fluid_gmres_iters=4, amg=amg))
    rr = o.solve(s.rhs, tol=1e-8)
    assert rr.converged and rr.true_relres <= 1e-8


@pytest.mark.parametrize("variant", ["lower", "upper", "diag"])
def test_exact_block_variants_are_their_triangular_solves(variant):
    """The block factorisations other than Alg. 2 (the remark after Sec. 4.1): with
    exact sub-solves "lower" is (D + L)^-1, "upper" (D + U)^-1 and "diag" D^-1,
    D = diag(M, S, F) and L (C_sm dropped) / U the strict block triangles."""
    s = tiny(2)
    A, I = _dense_blocks(s)
    D = np.zeros_like(A)
    L = np.zeros_like(A)
    U = np.zeros_like(A)
    for a in range(3):
        for b in range(3):
            blk = A[I[a], I[b]]
            if a == b:
                D[I[a], I[b]] = blk
            elif a > b and not (a == 1 and b == 0):
                L[I[a], I[b]] = blk
            elif a < b:
                U[I[a], I[b]] = blk
    P = {"lower": D + L, "upper": D + U, "diag": D}[variant]
    pre = oracle.BlockLDU(s.scipy(), s.offsets, 2, params=oracle.PrecondParams(variant=variant), exact=True)
    r = np.random.default_rng(8).standard_normal(A.shape[0])
    want = np.linalg.solve(P, r)
    assert np.allclose(pre(r), want, rtol=1e-9, atol=1e-9 * np.abs(want).max())
    # and each differs from Alg. 2 in the mesh block (Alg. 2's last step updates x_m)
    ldu = oracle.BlockLDU(s.scipy(), s.offsets, 2, exact=True)(r)
    m = I[0]
    assert np.linalg.norm(pre(r)[m] - ldu[m]) > 1e-6 * np.linalg.norm(ldu[m])


@pytest.mark.parametrize("variant", ["lower", "upper", "diag"])
def test_block_variants_converge_with_amg_subsolves(variant):
    s = tiny(2)
    o = oracle.OracleSolver.from_system(s, oracle.PrecondParams(mass_ratio=8.0, variant=variant))
    r = o.solve(s.rhs, tol=1e-8, restart=200)
    assert r.converged and r.true_relres <= 1e-8


@pytest.mark.parametrize("dim,theta", [(2, 0.5), (3, 0.51)])
def test_theta_scheme_systems_solve(dim, theta):
    """Crank-Nicolson (theta = 1/2) and shifted theta systems: the solid Schur
    coupling identity holds with c = dt*theta, and FGMRES with Alg. 2 reaches the
    tolerance when the preconditioner uses that c."""
    base = fsigen.CONFIGS["2d_tiny"].with_(name="cn2", n=(8, 8)) if dim == 2 else \
        fsigen.CONFIGS["3d"].with_(name="cn3", n=(4, 2, 4))
    cfg = base.with_(theta=theta)
    s = fsigen.make_system(cfg)
    prm = oracle.PrecondParams(mass_ratio=8.0 if dim == 2 else 20.0, dt_theta=cfg.dt * cfg.theta)
    pre = oracle.BlockLDU(s.scipy(), s.offsets, dim, params=prm)
    B = pre.B
    fixed_u = s.fixed[B.su]
    D = (B.A_uv + prm.dt_theta * B.A_uu).tocsr()
    assert abs(D[~fixed_u]).max() <= 1e-12 * abs(B.A_uu[~fixed_u]).max()
    r = oracle.OracleSolver.from_system(s, prm).solve(s.rhs, tol=1e-8)
    assert r.converged and r.true_relres <= 1e-8


@pytest.mark.parametrize("m", [1, 3])
def test_restarted_fgmres_cycles_are_krylov_minimisers(m):
    """Restarted FGMRES (Saad Alg. 9.6 with restart m) against what each cycle must
    return: with a fixed (linear) preconditioner M, cycle c moves x_c to the
    minimiser of ||b - A x|| over x_c + M K_m(A M, r_c), r_c = b - A x_c, computed
    here by least squares on an explicit (orthonormalised) Krylov basis; m = 1 is
    the minimal-residual step x + alpha M r.  Four cycles, so the update
    x = x_0 + Z y and the restart from the true residual are both exercised."""
    s = tiny(2)
    A = s.scipy()
    pre = oracle.BlockLDU(A, s.offsets, 2, params=params(2))
    b = s.rhs
    x = np.zeros(s.n)
    for c in range(4):
        r = b - A @ x
        K = [r / np.linalg.norm(r)]
        for _ in range(m - 1):
            K.append(A @ pre(K[-1]))
            K[-1] = K[-1] / np.linalg.norm(K[-1])
        Q, _ = np.linalg.qr(np.column_stack(K))
        Z = np.column_stack([pre(q) for q in Q.T])
        y, *_ = np.linalg.lstsq(A @ Z, r, rcond=None)
        x = x + Z @ y
        res = fgmres(lambda v: A @ v, pre, b, tol=1e-30, restart=m, maxit=(c + 1) * m)
        assert res.cycles == c + 1 and res.iters == (c + 1) * m
        assert np.linalg.norm(res.x - x) <= 1e-7 * np.linalg.norm(x), c
        # the residual estimate at the end of the cycle is the true residual of the update
        true = np.linalg.norm(b - A @ res.x) / np.linalg.norm(b)
        assert res.history[-1] == pytest.approx(true, rel=1e-6)
    # restarting never increases the residual (each cycle minimises over a space containing 0)
    ends = [np.linalg.norm(b - A @ fgmres(lambda v: A @ v, pre, b, tol=1e-30, restart=m, maxit=k * m).x)
            for k in range(1, 5)]
    assert np.all(np.diff(ends) <= 1e-12 * ends[0])


@pytest.mark.parametrize("dim", [2, 3])
def test_p1disc_systems_solve_like_dense_lu(dim):
    """Q2-Q2-P1disc Jacobians (the paper's pressure element, Sec. 3.4): no pressure
    rows couple to each other (C_pp = 0, so S_p = -B_pv diag(A_ff)^-1 B_vp), and
    FGMRES with Alg. 2 reaches the tolerance and the dense solution like the Q1 form."""
    cfg = (fsigen.CONFIGS["2d_tiny"].with_(name="pd2", n=(8, 8), pressure="p1disc") if dim == 2 else
           fsigen.CONFIGS["3d"].with_(name="pd3", n=(4, 2, 4), pressure="p1disc"))
    s = fsigen.make_system(cfg)
    B = oracle.Blocks(s.scipy(), s.offsets, dim)
    assert B.C_pp.nnz == 0
    S_p = oracle.pressure_schur(B).toarray()
    ref = -(B.B_pv @ np.diag(1.0 / B.A_ff.diagonal()) @ B.B_vp)
    assert np.allclose(S_p, ref, rtol=0, atol=1e-14 * np.abs(ref).max())
    xd = sla.solve(s.scipy().toarray(), s.rhs)
    o = oracle.OracleSolver.from_system(s, params(dim))
    r = o.solve(s.rhs, tol=1e-8)
    assert r.converged and r.true_relres <= 1e-8
    assert np.linalg.norm(r.x - xd) / np.linalg.norm(xd) <= np.linalg.cond(s.scipy().toarray(), 1) * 1e-8
