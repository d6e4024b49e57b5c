"""Pins of the seeded problem generator (input of the solve, Eq. mat:small).

The Jacobian is checked against its own residual by central differences, and
the residual/Jacobian against closed forms that the physics of Sec. 2-3 fixes:
Q2 mass integrals, Laplace stiffness annihilating linear fields, linear
elasticity annihilating rigid motions, frame invariance of the St. Venant-
Kirchhoff stress under a finite rotation, the discrete pressure gradient being
minus the transposed divergence, and the solid kinematic rows A_uv = -dt A_uu.
"""
from fractions import Fraction
import os

import numpy as np
import pytest
import scipy.sparse as sp

import fsigen

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def small(dim, n, **kw):
    base = fsigen.CONFIGS["2d_tiny"] if dim == 2 else fsigen.CONFIGS["3d"]
    return base.with_(name=f"t{dim}", n=n, **kw)


def A_of(pb, vals):
    return sp.csr_matrix((vals, pb.colind, pb.rowptr), shape=(pb.n, pb.n))


@pytest.mark.parametrize("name,expect", [
    ("2d_tiny", [0, 1584, 2178, 2772, 4356, 4645]),
    ("2d_mid", [0, 196992, 263682, 330372, 527364, 560517]),
    ("3d", [0, 154440, 212355, 270270, 424710, 434247]),
])
def test_dof_counts(name, expect):
    pb = fsigen.get_problem(fsigen.CONFIGS[name])
    assert pb.offsets.tolist() == expect


@pytest.mark.parametrize("cfg", [small(2, (8, 8)), small(2, (6, 4), prev_state="zero"), small(3, (4, 2, 4)),
                                 small(2, (8, 8), theta=0.5), small(3, (4, 2, 4), theta=0.51),
                                 small(2, (8, 8), pressure="p1disc"), small(3, (4, 2, 4), pressure="p1disc"),
                                 small(2, (6, 4), prev_state="zero", pressure="p1disc")])
def test_jacobian_matches_central_differences(cfg):
    pb = fsigen.get_problem(cfg)
    U = pb.seeded_state(3, 3e-2)
    Uold = U.copy() if cfg.prev_state == "rest" else None
    if Uold is not None:
        Uold = Uold * 0.5   # a previous step that differs from U exercises every term
    A = A_of(pb, pb.jacobian(U, Uold))
    rng = np.random.default_rng(7)
    for _ in range(3):
        d = rng.standard_normal(pb.n)
        d[pb.fixed] = 0.0
        eps = 1e-6
        fd = (pb.residual(U + eps * d, Uold) - pb.residual(U - eps * d, Uold)) / (2 * eps)
        ad = A @ d
        ad[pb.fixed] = 0.0
        assert np.linalg.norm(fd - ad) <= 1e-6 * np.linalg.norm(ad)


def test_q2_mass_integrals_solid_block():
    cfg = small(2, (8, 16))
    pb = fsigen.get_problem(cfg)
    A = A_of(pb, pb.jacobian(pb.seeded_state(), None))
    o = pb.offsets
    Auu = A[o[2]:o[3], o[2]:o[3]].tocsr()
    hx, hy = 2.0 / 8, 1.0 / 16
    gold = {}
    for line in open(os.path.join(GOLD, "q2_basis_integrals.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        gold[k] = float(Fraction(v))
    coords = pb.coords[o[2]:o[3]]
    comp = pb.comp[o[2]:o[3]]
    fixed = pb.fixed[o[2]:o[3]]
    ones = np.ones(Auu.shape[0])
    m1 = Auu @ ones
    checked = 0
    for i in range(Auu.shape[0]):
        x, y = coords[i]
        ix, iy = round(x / (hx / 2)), round(y / (hy / 2))
        # strictly inside the solid strip (y < 0.25) and away from fixed neighbours
        if fixed[i] or iy < 3 or iy > 5 or ix < 3 or ix > 13:
            continue
        kind = "vertex" if (ix % 2 == 0 and iy % 2 == 0) else ("center" if (ix % 2 and iy % 2) else "edge")
        assert m1[i] == pytest.approx(gold[kind] * hx * hy, rel=1e-12), (i, kind)
        checked += 1
    assert checked > 20


def test_mesh_block_annihilates_linear_fields_at_zero_state():
    cfg = small(2, (8, 8))
    pb = fsigen.get_problem(cfg)
    A = A_of(pb, pb.jacobian(np.zeros(pb.n), None))
    o = pb.offsets
    M = A[o[0]:o[1], o[0]:o[1]].tocsr()
    X = pb.coords[o[0]:o[1]]
    comp = pb.comp[o[0]:o[1]]
    field = 0.3 * X[:, 0] - 0.7 * X[:, 1] + 0.2     # affine, same for each component
    Mf = M @ field
    # rows whose whole Q2 neighbourhood is free and outside the solid closure
    hx, hy = 2.0 / 8, 1.0 / 8
    ix = np.rint(X[:, 0] / (hx / 2)).astype(int)
    iy = np.rint(X[:, 1] / (hy / 2)).astype(int)
    inner = (ix >= 3) & (ix <= 13) & (iy >= 7) & (iy <= 13)
    assert inner.sum() > 50
    scale = np.abs(M).max()
    assert np.max(np.abs(Mf[inner])) <= 1e-12 * scale


def test_linear_elasticity_kernel_rigid_modes_at_zero_state():
    cfg = small(2, (8, 16))
    pb = fsigen.get_problem(cfg)
    A = A_of(pb, pb.jacobian(np.zeros(pb.n), None))
    o = pb.offsets
    Avu = A[o[1]:o[2], o[2]:o[3]].tocsr()
    X = pb.coords[o[2]:o[3]]
    comp = pb.comp[o[2]:o[3]]
    hx, hy = 2.0 / 8, 1.0 / 16
    ix = np.rint(X[:, 0] / (hx / 2)).astype(int)
    iy = np.rint(X[:, 1] / (hy / 2)).astype(int)
    inner = (ix >= 3) & (ix <= 13) & (iy >= 3) & (iy <= 4)   # solid strip interior: y in (0, 0.25)
    assert inner.sum() > 20
    scale = np.abs(Avu).max()
    for mode in ("tx", "ty", "rot"):
        if mode == "tx":
            f = (comp == 0).astype(float)
        elif mode == "ty":
            f = (comp == 1).astype(float)
        else:
            f = np.where(comp == 0, -X[:, 1], X[:, 0])
        r = Avu @ f
        assert np.max(np.abs(r[inner])) <= 1e-11 * scale, mode


def test_stvk_frame_invariance_under_finite_rotation():
    """A rigid finite rotation u = (R - I) x has E = 0, so the solid stress rows and
    the mesh-motion rows (constant gradient, J = 1) see no force."""
    cfg = small(2, (8, 16))
    pb = fsigen.get_problem(cfg)
    ang = 0.3
    R = np.array([[np.cos(ang), -np.sin(ang)], [np.sin(ang), np.cos(ang)]])
    U = np.zeros(pb.n)
    u_rows = pb.field == 1
    X = pb.coords[u_rows]
    disp = X @ (R - np.eye(2)).T
    U[u_rows] = disp[np.arange(X.shape[0]), pb.comp[u_rows]]
    res = pb.residual(U, U.copy())
    o = pb.offsets
    hx, hy = 2.0 / 8, 1.0 / 16
    X = pb.coords
    ix = np.rint(X[:, 0] / (hx / 2)).astype(int)
    iy = np.rint(X[:, 1] / (hy / 2)).astype(int)
    sv = np.zeros(pb.n, bool)
    sv[o[1]:o[2]] = True
    inner_solid = sv & (ix >= 2) & (ix <= 14) & (iy >= 1) & (iy <= 6) & ~pb.fixed
    assert inner_solid.sum() > 20
    # the stress scale: dt * lambda * h ~ 2e6 * 0.01 * 0.06
    assert np.max(np.abs(res[inner_solid])) <= 1e-9 * (0.01 * 2e6 * hx)
    m = np.zeros(pb.n, bool)
    m[o[0]:o[1]] = True
    assert np.max(np.abs(res[m & ~pb.fixed])) <= 1e-12


@pytest.mark.parametrize("cfg", [small(2, (8, 8)), small(3, (4, 2, 4)), small(2, (8, 8), pressure="p1disc"),
                                 small(3, (4, 2, 4), pressure="p1disc")])
def test_pressure_gradient_is_minus_divergence_transpose(cfg):
    pb = fsigen.get_problem(cfg)
    U = pb.seeded_state(1, 3e-2)
    A = A_of(pb, pb.jacobian(U, U.copy()))
    o = pb.offsets
    Bvp = A[o[3]:o[4], o[4]:o[5]]
    Bpv = A[o[4]:o[5], o[3]:o[4]]
    D = (Bvp + Bpv.T)
    assert abs(D).max() <= 1e-13 * abs(Bvp).max()
    Bsp = A[o[1]:o[2], o[4]:o[5]]
    Bps = A[o[4]:o[5], o[1]:o[2]]
    assert abs(Bsp + Bps.T).max() <= 1e-13 * abs(Bsp).max()


@pytest.mark.parametrize("cfg", [small(2, (8, 8)), small(3, (4, 2, 4)), small(2, (8, 8), theta=0.5)])
def test_solid_kinematic_rows(cfg):
    """A_uv = -dt*theta*A_uu on the free kinematic rows (Sec. 4.3 mass identity)."""
    pb = fsigen.get_problem(cfg)
    U = pb.seeded_state(2, 3e-2)
    A = A_of(pb, pb.jacobian(U, U.copy()))
    o = pb.offsets
    Auv = A[o[2]:o[3], o[1]:o[2]]
    Auu = A[o[2]:o[3], o[2]:o[3]]
    free = ~pb.fixed[o[2]:o[3]]
    D = (Auv + cfg.dt * cfg.theta * Auu).tocsr()[free]
    assert abs(D).max() <= 1e-15 * abs(Auu).max()


@pytest.mark.parametrize("cfg", [small(2, (8, 8)), small(3, (4, 2, 4))])
def test_amg_blocks_structurally_symmetric(cfg):
    pb = fsigen.get_problem(cfg)
    o = pb.offsets
    P = sp.csr_matrix((np.ones(pb.nnz), pb.colind, pb.rowptr), shape=(pb.n, pb.n))
    for lo, hi in ((o[0], o[1]), (o[3], o[4])):
        B = P[lo:hi, lo:hi]
        assert (B != B.T).nnz == 0
    Svv = P[o[1]:o[2], o[1]:o[2]] + P[o[1]:o[2], o[2]:o[3]]
    assert (Svv != Svv.T).nnz == 0


def test_seeded_state_bounds_and_boundary():
    pb = fsigen.get_problem(small(2, (8, 8)))
    U = pb.seeded_state(0, 1e-2)
    assert np.max(np.abs(U)) <= 1e-2 + 1e-15
    X = pb.coords
    on = (X[:, 0] == 0) | (X[:, 1] == 0) | np.isclose(X[:, 0], 2.0) | np.isclose(X[:, 1], 1.0)
    assert np.max(np.abs(U[on])) <= 1e-15
    b1, b2 = pb.rhs(0), pb.rhs(0)
    assert np.array_equal(b1, b2) and np.all(b1[pb.fixed] == 0)


@pytest.mark.parametrize("dim,n", [(2, (8, 8)), (3, (4, 2, 4))])
@pytest.mark.parametrize("theta", [0.5, 0.51, 0.8])
def test_theta_scheme_at_rest_reduces_to_the_spatial_operator(dim, n, theta):
    """With the previous step equal to the state, every time-derivative term
    vanishes and the theta and (1 - theta) shares of each explicit-in-time term
    add up to one: R_theta(U, U) = R_1(U, U) for any theta (a missing or
    mis-weighted previous-level term breaks this)."""
    U = fsigen.get_problem(small(dim, n)).seeded_state(4, 3e-2)
    R1 = fsigen.get_problem(small(dim, n)).residual(U, U.copy())
    Rt = fsigen.get_problem(small(dim, n, theta=theta)).residual(U, U.copy())
    assert np.linalg.norm(Rt - R1) <= 1e-12 * np.linalg.norm(R1)


@pytest.mark.parametrize("dim,n", [(2, (8, 8)), (3, (4, 2, 4))])
def test_theta_scheme_jacobian_is_affine_in_theta_at_rest(dim, n):
    """At U = U_old the Jacobian is J_1 - (1 - theta) K with K the spatial part,
    so J_0.5 - J_1 = 2 (J_0.75 - J_1), and the two differ (K != 0)."""
    U = fsigen.get_problem(small(dim, n)).seeded_state(4, 3e-2)
    J = {t: fsigen.get_problem(small(dim, n, theta=t)).jacobian(U, U.copy()) for t in (1.0, 0.75, 0.5)}
    d1 = J[0.5] - J[1.0]
    d2 = J[0.75] - J[1.0]
    assert np.linalg.norm(d1 - 2.0 * d2) <= 1e-12 * np.linalg.norm(d1)
    assert np.linalg.norm(d1) > 1e-3 * np.linalg.norm(J[1.0])


@pytest.mark.parametrize("theta", [0.5, 0.8])
def test_theta_scheme_moving_previous_step(theta):
    """With U_old != U the previous level contributes: R_theta(U, U_old) differs
    from R_1 by (1 - theta) times the change of the explicit-in-time terms, i.e.
    R_theta is affine in theta at any (U, U_old)."""
    pbs = {t: fsigen.get_problem(small(2, (8, 8), theta=t)) for t in (1.0, theta, 0.5 * (1.0 + theta))}
    U = pbs[1.0].seeded_state(4, 3e-2)
    Uold = 0.5 * U
    R = {t: pb.residual(U, Uold) for t, pb in pbs.items()}
    mid = 0.5 * (1.0 + theta)
    assert np.linalg.norm(R[theta] - 2.0 * R[mid] + R[1.0]) <= 1e-11 * np.linalg.norm(R[1.0])
    assert np.linalg.norm(R[theta] - R[1.0]) > 1e-6 * np.linalg.norm(R[1.0])


@pytest.mark.parametrize("name,expect", [
    # Q2-Q2-P1disc: d + 1 pressure DOFs per fluid cell (16 x 12 = 192 in 2D, 32 x 16 x 12 in 3D)
    ("2d_tiny", [0, 1584, 2178, 2772, 4356, 4932]),
    ("3d", [0, 154440, 212355, 270270, 424710, 449286]),
])
def test_p1disc_dof_counts(name, expect):
    pb = fsigen.get_problem(fsigen.CONFIGS[name].with_(pressure="p1disc"))
    assert pb.offsets.tolist() == expect
    # every pressure row is a live row of one fluid cell (no identity rows)
    o = pb.offsets
    assert not pb.fixed[o[4]:o[5]].any()


@pytest.mark.parametrize("dim,n", [(2, (8, 8)), (3, (4, 4, 4))])
def test_p1disc_divergence_of_a_linear_field(dim, n):
    """Q2-Q2-P1disc (Sec. 3.4): at the state of rest (F = I, J = 1) the
    incompressibility rows are (div v, psi_k)_K with psi_0 = 1 and the centred
    linears psi_k = 2 xi_k - 1.  For a linear velocity field with divergence c
    (interpolated exactly by Q2 and integrated exactly by 3-point Gauss) row 0 of
    every fluid cell is c |K| and the linear rows vanish."""
    cfg = small(dim, n, pressure="p1disc")
    pb = fsigen.get_problem(cfg)
    z = np.zeros(pb.n)
    A = A_of(pb, pb.jacobian(z, z))
    o = pb.offsets
    v = np.zeros(pb.n)
    coef = [1.0, 0.5, -0.25][:dim]
    sel = (pb.field == 0)
    for i in range(dim):
        m = sel & (pb.comp == i)
        v[m] = coef[i] * pb.coords[m, i] + 0.3 * pb.coords[m, (i + 1) % dim]   # grad v has trace sum(coef)
    v[pb.fixed] = 0.0          # Dirichlet velocity rows are dropped columns: use interior cells only
    r = (A @ v)[o[4]:o[5]].reshape(-1, dim + 1)
    h = [cfg.L[d] / cfg.n[d] for d in range(dim)]
    vol = float(np.prod(h))
    c = sum(coef)
    # cells whose nodes are all free: pick by checking every node DOF of the cell is free
    cd, cf = pb.cell_map()
    fluid = (cf & 1) == 0
    nq2 = 9 if dim == 2 else 27
    vdofs = cd[:, :nq2 * dim]
    interior = fluid & ~pb.fixed[vdofs].any(axis=1)
    assert interior.sum() > 0
    pdof0 = cd[interior, 2 * nq2 * dim]
    rows = (pdof0 - o[4]) // (dim + 1)
    np.testing.assert_allclose(r[rows, 0], c * vol, rtol=1e-12)
    assert np.max(np.abs(r[rows, 1:])) <= 1e-12 * vol


def test_p1disc_has_no_learned_node_map():
    pb = fsigen.get_problem(small(2, (8, 8), pressure="p1disc"))
    with pytest.raises(ValueError):
        pb.node_map()
