"""Parity of the CUDA solver (through the C ABI) with the FP64 CPU oracle on
seeded FSI Jacobians: outer SpMV, every AMG level (aggregates bit-exact,
lambda, Galerkin matrices), every block inverse of Alg. 2, and whole FGMRES
solves in the FP64 and FP32-AMG forms.

Tolerances: FP64 pieces agree to rounding (1e-11 relative; the oracle sums in
another order); FP64 solves agree with the oracle's to 1e-8 relative solution
error with iteration counts within +-1.  The FP32-AMG form runs another Krylov
trajectory; both stop at ||b - Ax||/||b|| <= 1e-8, and with condition numbers
near 1e14 that residual bounds the solution error only to ~1e-2 (measured: the
FP64 oracle solution is 7e-3 from the manufactured x* on the 64x32 mesh, almost
all of it in the pressure).  The FP32 form is therefore required to meet the
1e-8 residual and to be as accurate as the FP64 form: error against x* within
10x of the FP64 oracle's error (1e-6 when that is smaller)."""
import numpy as np
import pytest
import scipy.sparse as sp

import fsigen
import oracle

pytestmark = pytest.mark.gpu

CASES = {
    "2d_16x16": (fsigen.CONFIGS["2d_tiny"], 8.0),
    "2d_64x32": (fsigen.CONFIGS["2d_tiny"].with_(name="2d_64x32", n=(64, 32)), 8.0),
    "2d_37x19_ragged": (fsigen.CONFIGS["2d_tiny"].with_(name="2d_37x19", n=(37, 19), state_seed=3, rhs_seed=5), 8.0),
    "3d_8x4x4": (fsigen.CONFIGS["3d"].with_(name="3d_8x4x4", n=(8, 4, 4)), 20.0),
}
HIER = ["mesh", "solid_schur", "fluid_velocity", "pressure_schur"]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_05648_gb300 import build
    build.build()
    return torch


_cache = {}


def case(name, torch):
    if name not in _cache:
        import paper_1801_05648_gb300 as P
        cfg, mr = CASES[name]
        s = fsigen.make_system(cfg)
        o = oracle.OracleSolver.from_system(s, params=oracle.PrecondParams(mass_ratio=mr))
        ref = o.solve(s.rhs)
        g = P.FSISolver.from_system(s, params=P.default_params(s.dim, mass_ratio=mr))
        g.precond_build("fp64")
        _cache[name] = (s, o, ref, g, mr)
    return _cache[name]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name", list(CASES))
def test_operator_parity(name, torch_cuda):
    torch = torch_cuda
    s, o, ref, g, _ = case(name, torch)
    x = np.random.default_rng(11).standard_normal(s.n)
    xt = torch.tensor(x, device="cuda")
    yt = torch.empty_like(xt)
    g.apply_operator(xt, yt)
    assert rel(yt.cpu().numpy(), s.scipy() @ x) <= 1e-13


@pytest.mark.parametrize("name", list(CASES))
def test_hierarchies_match_oracle(name, torch_cuda):
    s, o, ref, g, _ = case(name, torch_cuda)
    invs = [o.P.M_inv, o.P.Shat_inv, o.P.Aff_inv, o.P.Sp_inv]
    for w, inv in enumerate(invs):
        H = inv.H
        info = g.amg_info(w, 0)
        assert info["levels"] == len(H.levels), HIER[w]
        for lvl in range(len(H.levels)):
            li = g.amg_info(w, lvl)
            assert li["lam"] == pytest.approx(H.levels[lvl].lam, rel=1e-12)
            if lvl + 1 < len(H.levels):
                assert np.array_equal(g.amg_export(w, lvl, "agg"), H.levels[lvl].agg), (HIER[w], lvl)
            if lvl > 0:
                rp, ci, va = g.amg_export(w, lvl, "A")
                b = li["b"]
                Ag = sp.bsr_matrix((va, ci, rp), shape=(li["nbrows"] * b,) * 2).toarray()
                Ao = H.levels[lvl].A.toarray()
                assert np.linalg.norm(Ag - Ao) <= 1e-12 * np.linalg.norm(Ao), (HIER[w], lvl)


def _block_slices(s, o):
    of = s.offsets
    return [("mesh", slice(of[0], of[1]), o.P.M_inv), ("solid_schur", slice(of[1], of[2]), o.P.Shat_inv),
            ("fluid_velocity", slice(of[3], of[4]), o.P.Aff_inv), ("pressure_schur", slice(of[4], of[5]), o.P.Sp_inv),
            ("solid_mass", slice(of[2], of[3]), o.P.Ms_inv), ("solid", slice(of[1], of[3]), o.P.S_inv),
            ("fluid", slice(of[3], of[5]), o.P.F_inv), ("precond", slice(0, s.n), o.P)]


@pytest.mark.parametrize("name", list(CASES))
def test_block_inverses_fp64(name, torch_cuda):
    torch = torch_cuda
    s, o, ref, g, _ = case(name, torch)
    for blk, sl, f in _block_slices(s, o):
        r = np.random.default_rng(3).standard_normal(sl.stop - sl.start)
        rt = torch.tensor(r, device="cuda")
        zt = torch.zeros_like(rt)
        g.apply_block(blk, rt, zt)
        assert rel(zt.cpu().numpy(), f(r)) <= 1e-11, blk


@pytest.mark.parametrize("name", list(CASES))
def test_solve_fp64_parity(name, torch_cuda):
    torch = torch_cuda
    s, o, ref, g, _ = case(name, torch)
    b = torch.tensor(s.rhs, device="cuda")
    x = torch.zeros_like(b)
    st = g.solve(b, x, 1e-8)
    xc = x.cpu().numpy()
    assert st.status == 0 and st.true_relres <= 1e-8
    assert np.linalg.norm(s.rhs - s.scipy() @ xc) / np.linalg.norm(s.rhs) <= 1e-8 * 1.001
    assert abs(st.iters - ref.iters) <= 1, (st.iters, ref.iters)
    assert rel(xc, ref.x) <= 1e-8
    # residual history: monotone within each cycle, last estimate below tol
    assert st.history[-1] <= 1e-8 and len(st.history) == st.iters
    # the GPU orthogonalises the defect v_j - A z_j (one Gram-Schmidt pass unless it
    # keeps < 1% of the norm), the oracle A z_j by CGS2: the same Arnoldi vectors in
    # exact arithmetic, so the Givens residual estimates agree to rounding
    assert 0 <= st.reorth_passes <= st.iters
    if st.iters == ref.iters:
        h, hr = np.array(st.history), np.array(ref.history)
        assert np.all(np.abs(h - hr) <= 1e-6 * hr), np.abs(h / hr - 1).max()


@pytest.mark.parametrize("name", list(CASES))
def test_solve_fp32_amg(name, torch_cuda):
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    s, o, ref, _, mr = case(name, torch)
    g = P.FSISolver.from_system(s, params=P.default_params(s.dim, mass_ratio=mr))
    g.precond_build("fp32")
    b = torch.tensor(s.rhs, device="cuda")
    x = torch.zeros_like(b)
    st = g.solve(b, x, 1e-8)
    xc = x.cpu().numpy()
    assert st.status == 0 and st.true_relres <= 1e-8
    assert np.linalg.norm(s.rhs - s.scipy() @ xc) / np.linalg.norm(s.rhs) <= 1e-8 * 1.001
    err64 = rel(ref.x, s.x_exact)
    assert rel(xc, s.x_exact) <= max(10.0 * err64, 1e-6), (rel(xc, s.x_exact), err64)
    # FP32 block inverses agree with the FP64 oracle to single precision
    for blk, sl, f in _block_slices(s, o):
        r = np.random.default_rng(3).standard_normal(sl.stop - sl.start)
        rt = torch.tensor(r, device="cuda")
        zt = torch.zeros_like(rt)
        g.apply_block(blk, rt, zt)
        assert rel(zt.cpu().numpy(), f(r)) <= 1e-4, blk
    g.close()


def test_graph_replay_is_bit_identical(torch_cuda):
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    s, o, ref, _, mr = case("2d_64x32", torch)
    b = torch.tensor(s.rhs, device="cuda")
    xs = []
    for flags in (0, P.FSI_USE_GRAPHS):
        for prec in ("fp64", "fp32"):
            g = P.FSISolver.from_system(s, params=P.default_params(2, flags=flags))
            g.precond_build(prec)
            x = torch.zeros_like(b)
            st = g.solve(b, x, 1e-8)
            x2 = torch.zeros_like(b)
            st2 = g.solve(b, x2, 1e-8)          # second solve reuses the captured graph
            assert torch.equal(x, x2) and st.iters == st2.iters
            xs.append(x.cpu().numpy())
            g.close()
    assert np.array_equal(xs[0], xs[2]) and np.array_equal(xs[1], xs[3])


def test_launch_modes_are_bit_identical(torch_cuda):
    """Programmatic dependent launch on/off and the SpMV prefetch modes change only
    launch attributes and the assignment of rows to CTAs: every solve is bit-identical.
    (The knobs belong to the context: each call applies its own context's values.)"""
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    s, o, ref, _, mr = case("2d_64x32", torch)
    b = torch.tensor(s.rhs, device="cuda")
    G = P.FSI_USE_GRAPHS
    modes = [dict(flags=G), dict(flags=G | P.FSI_NO_PDL), dict(flags=G, spmv_prefetch=0),
             dict(flags=G, spmv_prefetch=2), dict(flags=0, spmv_prefetch=0)]
    for prec in ("fp64", "fp32"):
        first = None
        for kw in modes:
            g = P.FSISolver.from_system(s, params=P.default_params(2, **kw))
            g.precond_build(prec)
            x = torch.zeros_like(b)
            st = g.solve(b, x, 1e-8)
            g.close()
            if first is None:
                first = (x, st.iters)
            else:
                assert torch.equal(x, first[0]) and st.iters == first[1], (prec, kw)


def test_staged_chebyshev_is_bit_identical(torch_cuda):
    """The opt-in staged 2 x 2 FP32 Chebyshev kernel (persistent CTAs, column offsets
    copied into shared memory by the TMA engine one chunk ahead) visits every block in
    the order of the default kernel: FP32-AMG solves on 512x256 (level 0 of the mesh and
    fluid hierarchies: 6,150 chunks, enough for the persistent grid) are bit-identical."""
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    s = fsigen.make_system(fsigen.CONFIGS["2d_512x256"])
    b = torch.tensor(s.rhs, device="cuda")
    out = []
    for stage in (0, 1):
        g = P.FSISolver.from_system(s, params=P.default_params(2, flags=P.FSI_USE_GRAPHS, spmv_stage=stage))
        g.precond_build("fp32")
        x = torch.zeros_like(b)
        st = g.solve(b, x, 1e-8)
        g.close()
        assert st.status == 0
        out.append((x, st.iters, st.history))
    assert out[0][1] == out[1][1] and out[0][2] == out[1][2]
    assert torch.equal(out[0][0], out[1][0])


@pytest.mark.parametrize("name", ["2d_37x19_ragged", "3d_8x4x4", "2d_512x256"])
def test_length_ordered_rows_are_bit_identical(name, torch_cuda):
    """spmv_order only changes which thread sums a block row of the outer operator
    (rows sorted by length within 32-row windows, ragged last windows included), never
    the order of a row's sum: the operator, its residual and whole FP64 and FP32-AMG
    solves with and without it are bit-identical (2D and 3D)."""
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    cfg = fsigen.CONFIGS["2d_512x256"] if name == "2d_512x256" else CASES[name][0]
    s = fsigen.make_system(cfg)
    b = torch.tensor(s.rhs, device="cuda")
    xr = torch.tensor(np.random.default_rng(7).standard_normal(s.n), device="cuda")
    for prec in ("fp64", "fp32"):
        out = []
        for order in (0, 1):
            g = P.FSISolver.from_system(s, params=P.default_params(s.dim, flags=P.FSI_USE_GRAPHS, spmv_order=order))
            g.precond_build(prec)
            y = torch.empty_like(b)
            g.apply_operator(xr, y)
            x = torch.zeros_like(b)
            st = g.solve(b, x, 1e-8)
            g.close()
            assert st.status == 0
            out.append((x, st.iters, st.history, y))
        assert out[0][1] == out[1][1] and out[0][2] == out[1][2], prec
        assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][3], out[1][3]), prec
        if prec == "fp64":
            A = s.scipy()
            want = A @ xr.cpu().numpy()
            assert np.abs(out[1][3].cpu().numpy() - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("deg", [0, 1, 3])
def test_coarse_chebyshev_degree_parity(deg, torch_cuda):
    """The coarse-level Chebyshev degree (0: the level-0 degree everywhere) is the
    same algorithm on both sides: FP64 solves agree like the default ones."""
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    cfg, mr = CASES["2d_64x32"]
    s = fsigen.make_system(cfg)
    o = oracle.OracleSolver.from_system(
        s, params=oracle.PrecondParams(mass_ratio=mr, amg=oracle.AMGParams(cheb_degree_coarse=deg)))
    ref = o.solve(s.rhs)
    g = P.FSISolver.from_system(s, params=P.default_params(2, mass_ratio=mr, cheb_degree_coarse=deg))
    g.precond_build("fp64")
    b = torch.tensor(s.rhs, device="cuda")
    x = torch.zeros_like(b)
    st = g.solve(b, x, 1e-8)
    g.close()
    assert st.status == 0 and abs(st.iters - ref.iters) <= 1, (st.iters, ref.iters)
    assert rel(x.cpu().numpy(), ref.x) <= 1e-8


def test_edge_cases(torch_cuda):
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    s, o, ref, g, mr = case("2d_16x16", torch)
    z = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    x = torch.full_like(z, 7.0)
    st = g.solve(z, x, 1e-8)                       # zero right-hand side: x = 0, no iterations
    assert st.status == 0 and st.iters == 0 and torch.count_nonzero(x).item() == 0
    bad = torch.tensor(s.rhs, device="cuda")
    bad[5] = float("nan")
    with pytest.raises(P.FSIError) as e:
        g.solve(bad, x, 1e-8)
    assert e.value.code == -6
    g3 = P.FSISolver.from_system(s, params=P.default_params(2, maxit=3))
    g3.precond_build("fp64")
    b = torch.tensor(s.rhs, device="cuda")
    st = g3.solve(b, x, 1e-8, raise_on_error=False)
    assert st.status == -4 and st.iters == 3 and 0 < st.true_relres < 1
    g3.close()
    # warm start from the converged solution: no iteration needed
    gw = P.FSISolver.from_system(s, params=P.default_params(2, flags=P.FSI_X0_GIVEN))
    gw.precond_build("fp64")
    x0 = torch.tensor(ref.x, device="cuda")
    st = gw.solve(b, x0, 1e-8)
    assert st.status == 0 and st.iters == 0
    # precond before build is refused
    gn = P.FSISolver.from_system(s)
    with pytest.raises(P.FSIError):
        gn.solve(b, x, 1e-8)
    gw.close(); gn.close()


@pytest.mark.parametrize("name,theta", [("2d_16x16", 0.5), ("3d_8x4x4", 0.51)])
def test_theta_scheme_parity(name, theta, torch_cuda):
    """Jacobians of the theta scheme (Crank-Nicolson, shifted): with
    dt_theta = dt*theta in both, P^-1 in FP64 matches the oracle to 1e-11 and the
    FP64 solve to 1e-8 within one iteration; the FP32-AMG form meets the residual."""
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    cfg0, mr = CASES[name]
    cfg = cfg0.with_(theta=theta)
    s = fsigen.make_system(cfg)
    c = cfg.dt * cfg.theta
    o = oracle.OracleSolver.from_system(s, params=oracle.PrecondParams(mass_ratio=mr, dt_theta=c))
    ref = o.solve(s.rhs)
    b = torch.tensor(s.rhs, device="cuda")
    for prec in ("fp64", "fp32"):
        g = P.FSISolver.from_system(s, params=P.default_params(s.dim, mass_ratio=mr, dt_theta=c,
                                                               flags=P.FSI_USE_GRAPHS))
        g.precond_build(prec)
        if prec == "fp64":
            r = np.random.default_rng(3).standard_normal(s.n)
            rt = torch.tensor(r, device="cuda")
            zt = torch.zeros_like(rt)
            g.apply_block("precond", rt, zt)
            assert rel(zt.cpu().numpy(), o.P(r)) <= 1e-11
        x = torch.zeros_like(b)
        st = g.solve(b, x, 1e-8)
        g.close()
        xc = x.cpu().numpy()
        assert st.status == 0
        assert np.linalg.norm(s.rhs - s.scipy() @ xc) / np.linalg.norm(s.rhs) <= 1e-8 * 1.001
        if prec == "fp64":
            assert abs(st.iters - ref.iters) <= 1 and rel(xc, ref.x) <= 1e-8


@pytest.mark.parametrize("variant", ["lower", "upper", "diag"])
@pytest.mark.parametrize("name", ["2d_37x19_ragged", "3d_8x4x4"])
def test_block_factorisation_variants(name, variant, torch_cuda):
    """precond_variant (the block orderings of the remark after Sec. 4.1): P^-1 in
    FP64 against the oracle's variant to 1e-11, the FP64 solve within 1 iteration
    and 1e-8 of the oracle's, and the FP32-AMG solve to the residual."""
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    code = {"lower": P.FSI_PRECOND_LOWER, "upper": P.FSI_PRECOND_UPPER, "diag": P.FSI_PRECOND_DIAG}[variant]
    cfg, mr = CASES[name]
    s = fsigen.make_system(cfg)
    o = oracle.OracleSolver.from_system(s, params=oracle.PrecondParams(mass_ratio=mr, variant=variant))
    ref = o.solve(s.rhs)
    b = torch.tensor(s.rhs, device="cuda")
    for prec in ("fp64", "fp32"):
        g = P.FSISolver.from_system(s, params=P.default_params(s.dim, mass_ratio=mr, flags=P.FSI_USE_GRAPHS,
                                                               precond_variant=code))
        g.precond_build(prec)
        if prec == "fp64":
            r = np.random.default_rng(3).standard_normal(s.n)
            rt = torch.tensor(r, device="cuda")
            zt = torch.zeros_like(rt)
            g.apply_block("precond", rt, zt)
            assert rel(zt.cpu().numpy(), o.P(r)) <= 1e-11
        x = torch.zeros_like(b)
        st = g.solve(b, x, 1e-8)
        g.close()
        xc = x.cpu().numpy()
        assert st.status == 0
        assert np.linalg.norm(s.rhs - s.scipy() @ xc) / np.linalg.norm(s.rhs) <= 1e-8 * 1.001
        if prec == "fp64":
            assert abs(st.iters - ref.iters) <= 1 and rel(xc, ref.x) <= 1e-8


@pytest.mark.parametrize("name", ["2d_16x16", "2d_37x19_ragged", "3d_8x4x4"])
def test_fluid_inner_gmres_parity(name, torch_cuda):
    """FSI_FLUID_GMRES (Sec. 4.4): every A_ff^-1 of the fluid solve is k = 4 steps of
    V-cycle-preconditioned GMRES.  FP64 against the oracle's fluid_gmres_iters = 4:
    the A_ff, fluid and Alg. 2 applications to rounding (GMRES keeps the V-cycle's
    1e-11 up to the growth of its k steps), the solve to 1e-8 with the iteration
    count within +-1; switching the flag on an existing context re-captures the
    iteration graph; the FP32-AMG form meets the residual and the error bound."""
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    cfg, mr = CASES[name]
    s = fsigen.make_system(cfg)
    op = oracle.PrecondParams(mass_ratio=mr, fluid_gmres_iters=4)
    o = oracle.OracleSolver.from_system(s, params=op)
    ref = o.solve(s.rhs)
    G = P.FSI_USE_GRAPHS
    g = P.FSISolver.from_system(s, params=P.default_params(s.dim, mass_ratio=mr, flags=G | P.FSI_FLUID_GMRES,
                                                           fluid_gmres_iters=4))
    g.precond_build("fp64")
    for blk, sl, f in _block_slices(s, o):
        if blk not in ("fluid_velocity", "fluid", "precond"):
            continue
        r = np.random.default_rng(3).standard_normal(sl.stop - sl.start)
        rt = torch.tensor(r, device="cuda")
        zt = torch.zeros_like(rt)
        g.apply_block(blk, rt, zt)
        assert rel(zt.cpu().numpy(), f(r)) <= 1e-10, blk
    b = torch.tensor(s.rhs, device="cuda")
    x = torch.zeros_like(b)
    st = g.solve(b, x, 1e-8)
    assert st.status == 0 and st.true_relres <= 1e-8
    assert abs(st.iters - ref.iters) <= 1 and rel(x.cpu().numpy(), ref.x) <= 1e-8
    # the same context with the flag off solves like the plain form, and on again like above
    _, _, ref0, _, _ = case(name, torch)
    g.set_flags(G)
    x0 = torch.zeros_like(b)
    st0 = g.solve(b, x0, 1e-8)
    assert abs(st0.iters - ref0.iters) <= 1 and rel(x0.cpu().numpy(), ref0.x) <= 1e-8
    g.set_flags(G | P.FSI_FLUID_GMRES)
    x1 = torch.zeros_like(b)
    st1 = g.solve(b, x1, 1e-8)
    assert st1.iters == st.iters and np.array_equal(x1.cpu().numpy(), x.cpu().numpy())
    g.close()
    g32 = P.FSISolver.from_system(s, params=P.default_params(s.dim, mass_ratio=mr, flags=G | P.FSI_FLUID_GMRES,
                                                             fluid_gmres_iters=4))
    g32.precond_build("fp32")
    x32 = torch.zeros_like(b)
    st32 = g32.solve(b, x32, 1e-8)
    g32.close()
    xc = x32.cpu().numpy()
    assert st32.status == 0
    assert np.linalg.norm(s.rhs - s.scipy() @ xc) / np.linalg.norm(s.rhs) <= 1e-8 * 1.001
    e64 = rel(ref.x, s.x_exact)
    assert rel(xc, s.x_exact) <= max(10.0 * e64, 1e-6)


@pytest.mark.parametrize("name", ["2d_mid", "3d", "2d_large"])
def test_full_size_solves(name, torch_cuda):
    """Full-size Jacobians: the solve reaches 1e-8 confirmed by an FP64 CPU residual,
    sampled operator rows match, and the FP32-AMG form is as accurate (against the
    manufactured solution) as the FP64 form."""
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    s = fsigen.make_system(name)
    A = s.scipy()
    mr = 8.0 if s.dim == 2 else 20.0
    b = torch.tensor(s.rhs, device="cuda")
    xs = {}
    for prec in ("fp64", "fp32"):
        g = P.FSISolver.from_system(s, params=P.default_params(s.dim, mass_ratio=mr, flags=P.FSI_USE_GRAPHS))
        g.precond_build(prec)
        x = torch.zeros_like(b)
        st = g.solve(b, x, 1e-8)
        xc = x.cpu().numpy()
        assert st.status == 0
        assert np.linalg.norm(s.rhs - A @ xc) / np.linalg.norm(s.rhs) <= 1e-8 * 1.001
        xs[prec] = xc
        if prec == "fp64":
            rows = np.sort(np.random.default_rng(2).choice(s.n, 2000, replace=False))
            v = np.random.default_rng(4).standard_normal(s.n)
            vt = torch.tensor(v, device="cuda")
            yt = torch.empty_like(vt)
            g.apply_operator(vt, yt)
            yr = A[rows] @ v
            assert np.max(np.abs(yt.cpu().numpy()[rows] - yr)) <= 1e-12 * np.max(np.abs(yr))
        g.close()
    e64, e32 = rel(xs["fp64"], s.x_exact), rel(xs["fp32"], s.x_exact)
    assert e32 <= max(10.0 * e64, 1e-6), (e32, e64)


@pytest.mark.parametrize("name", ["2d_16x16", "2d_64x32", "3d_8x4x4"])
@pytest.mark.parametrize("mode", ["cluster", "grid"])
def test_coarse_vcycle_in_one_launch_matches_per_level_path(name, mode, torch_cuda):
    """FSI_CLUSTER_COARSE / FSI_GRID_COARSE run the coarse levels of each V-cycle in one
    launch (a thread-block cluster, or a cooperative grid with a software barrier); the
    block inverses and the solve must match the oracle like the per-level path."""
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    s, o, ref, g, mr = case(name, torch)
    flag = P.FSI_CLUSTER_COARSE if mode == "cluster" else P.FSI_GRID_COARSE
    for prec, tol in (("fp64", 1e-11), ("fp32", 1e-4)):
        gc = P.FSISolver.from_system(s, params=P.default_params(s.dim, mass_ratio=mr, flags=flag))
        gc.precond_build(prec)
        for blk, sl, f in _block_slices(s, o):
            r = np.random.default_rng(3).standard_normal(sl.stop - sl.start)
            rt = torch.tensor(r, device="cuda")
            zt = torch.zeros_like(rt)
            gc.apply_block(blk, rt, zt)
            assert rel(zt.cpu().numpy(), f(r)) <= tol, (prec, blk)
        b = torch.tensor(s.rhs, device="cuda")
        x = torch.zeros_like(b)
        st = gc.solve(b, x, 1e-8)
        assert st.status == 0 and st.true_relres <= 1e-8
        if prec == "fp64":
            assert abs(st.iters - ref.iters) <= 1 and rel(x.cpu().numpy(), ref.x) <= 1e-8
        gc.close()


@pytest.mark.parametrize("name,m", [("2d_16x16", 2), ("2d_37x19_ragged", 3), ("3d_8x4x4", 2)])
def test_restart_cycles_match_oracle(name, m, torch_cuda):
    """FGMRES(m) with restarts (Saad Alg. 9.6): each cycle ends at j = m (or at the
    tolerance), x = x_0 + Z y is formed, the true residual recomputed and a new
    Arnoldi basis started.  With the same m the FP64 GPU solve follows the oracle's:
    the same number of cycles, iterations within +-1, solution within 1e-8; the
    FP32-AMG form restarts the same way and meets the residual."""
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    cfg, mr = CASES[name]
    s = fsigen.make_system(cfg)
    o = oracle.OracleSolver.from_system(s, params=oracle.PrecondParams(mass_ratio=mr))
    ref = o.solve(s.rhs, restart=m)
    assert ref.converged and ref.cycles >= 2
    b = torch.tensor(s.rhs, device="cuda")
    for prec in ("fp64", "fp32"):
        for flags in (0, P.FSI_USE_GRAPHS):
            g = P.FSISolver.from_system(s, params=P.default_params(s.dim, mass_ratio=mr, restart=m, flags=flags))
            g.precond_build(prec)
            x = torch.zeros_like(b)
            st = g.solve(b, x, 1e-8)
            g.close()
            xc = x.cpu().numpy()
            assert st.status == 0 and st.cycles >= 2, (prec, st.cycles)
            assert np.linalg.norm(s.rhs - s.scipy() @ xc) / np.linalg.norm(s.rhs) <= 1e-8 * 1.001
            if prec == "fp64":
                assert st.cycles == ref.cycles and abs(st.iters - ref.iters) <= 1, (st.cycles, ref.cycles, st.iters)
                assert rel(xc, ref.x) <= 1e-8


@pytest.mark.parametrize("name,states", [("2d_mid", [0, 1, 2, 3, 4]), ("3d", [0])])
def test_full_size_fp64_matches_oracle(name, states, torch_cuda):
    """Element-wise parity at the full sizes of the 256x128 (five seeded states) and
    32x16x16 workloads: the FP64 GPU solve against the FP64 oracle's solve of the
    same Jacobian (same hierarchy up to rounding, aggregates bit-exact), relative
    solution error <= 1e-8 and iteration counts within +-1."""
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    for st_seed in states:
        s = fsigen.make_system(fsigen.CONFIGS[name].with_(state_seed=st_seed))
        mr = 8.0 if s.dim == 2 else 20.0
        ref = oracle.OracleSolver.from_system(s, params=oracle.PrecondParams(mass_ratio=mr)).solve(s.rhs)
        assert ref.converged
        g = P.FSISolver.from_system(s, params=P.default_params(s.dim, mass_ratio=mr, flags=P.FSI_USE_GRAPHS))
        g.precond_build("fp64")
        b = torch.tensor(s.rhs, device="cuda")
        x = torch.zeros_like(b)
        st = g.solve(b, x, 1e-8)
        g.close()
        xc = x.cpu().numpy()
        e = rel(xc, ref.x)
        print(f"[parity] {name} state {st_seed}: GPU FP64 {st.iters} it, oracle {ref.iters} it, "
              f"rel. difference {e:.3e}")
        assert st.status == 0 and abs(st.iters - ref.iters) <= 1, (st_seed, st.iters, ref.iters)
        assert e <= 1e-8, (st_seed, e)


@pytest.mark.parametrize("name", ["2d_16x16", "2d_64x32"])
def test_mixed_forms_against_tightened_oracle(name, torch_cuda):
    """Accuracy of every form against an oracle solve tightened to rtol 1e-12 (the
    reference).  These Jacobians have condition numbers near 1e14 (16x16: 2.1e14 in
    the 2-norm), so a residual of 1e-8 fixes the solution only to ~1e-3 and even a
    sparse direct solve lies ~1e-4 from the reference: a form is held to what the
    FP64 oracle itself reaches at the same tolerance (within 10x of the oracle's
    own distance from the reference, or 1e-6 when that is larger).  Checked at
    rtol 1e-8 (the workloads' tolerance) and 1e-11 for the FP64, FP32-AMG and
    FP32-AMG + learned-stage forms."""
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    import os
    cfg, mr = CASES[name]
    s = fsigen.make_system(cfg)
    o = oracle.OracleSolver.from_system(s, params=oracle.PrecondParams(mass_ratio=mr))
    ref = o.solve(s.rhs, tol=1e-12, restart=200)
    assert ref.converged
    pb = fsigen.get_problem(s.cfg)
    nd, pt = pb.node_map()
    wpath = os.path.join(os.path.dirname(P.__file__), "weights", "mlp_fsi2d_256x128.bin")
    b = torch.tensor(s.rhs, device="cuda")
    for tol in (1e-8, 1e-11):
        yard = rel(o.solve(s.rhs, tol=tol, restart=200).x, ref.x)
        for form in ("fp64", "fp32", "learned"):
            g = P.FSISolver.from_system(s, params=P.default_params(2, mass_ratio=mr, restart=200,
                                                                   flags=P.FSI_USE_GRAPHS))
            g.precond_build("fp64" if form == "fp64" else "fp32")
            if form == "learned":
                g.learned_setup(nd, pt)
                g.learned_load(wpath)
                g.set_flags(P.FSI_USE_GRAPHS | P.FSI_LEARNED)
            x = torch.zeros_like(b)
            st = g.solve(b, x, tol)
            g.close()
            e = rel(x.cpu().numpy(), ref.x)
            print(f"[accuracy] {name} rtol {tol:.0e} {form}: {st.iters} it, vs oracle(1e-12) {e:.3e}; "
                  f"oracle at the same rtol {yard:.3e}")
            assert st.status == 0
            assert e <= max(10.0 * yard, 1e-6), (tol, form, e, yard)


def test_short_tensors_are_refused(torch_cuda):
    """The binding checks every device vector's length before handing its address to
    the library (a short tensor would be read or written past its end)."""
    torch = torch_cuda
    s, o, ref, g, _ = case("2d_16x16", torch)
    short = torch.zeros(s.n - 1, dtype=torch.float64, device="cuda")
    full = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        g.solve(short, full, 1e-8)
    with pytest.raises(ValueError):
        g.apply_operator(full, short)
    n_m = int(s.offsets[1] - s.offsets[0])
    with pytest.raises(ValueError):
        g.apply_block("mesh", full[:n_m - 1], full[:n_m])
    with pytest.raises(ValueError):
        g.mass_solve_noalloc(full[:3], full[:3])


@pytest.mark.parametrize("cfg", [fsigen.CONFIGS["2d_tiny"].with_(name="pd16", pressure="p1disc"),
                                 fsigen.CONFIGS["2d_tiny"].with_(name="pd37", n=(37, 19), state_seed=3, rhs_seed=5,
                                                                 pressure="p1disc"),
                                 fsigen.CONFIGS["3d"].with_(name="pd3", n=(8, 4, 4), pressure="p1disc")],
                         ids=["2d_16x16", "2d_37x19_ragged", "3d_8x4x4"])
def test_p1disc_parity(cfg, torch_cuda):
    """Q2-Q2-P1disc Jacobians (Sec. 3.4): the same solver, unchanged, on the paper's
    pressure element.  P^-1 in FP64 against the oracle to 1e-11, the FP64 solve within
    1e-8 and one iteration of the oracle's, the FP32-AMG form to the residual."""
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    s = fsigen.make_system(cfg)
    mr = 8.0 if s.dim == 2 else 20.0
    o = oracle.OracleSolver.from_system(s, params=oracle.PrecondParams(mass_ratio=mr))
    ref = o.solve(s.rhs)
    b = torch.tensor(s.rhs, device="cuda")
    for prec in ("fp64", "fp32"):
        g = P.FSISolver.from_system(s, params=P.default_params(s.dim, mass_ratio=mr, flags=P.FSI_USE_GRAPHS))
        g.precond_build(prec)
        if prec == "fp64":
            r = np.random.default_rng(3).standard_normal(s.n)
            rt = torch.tensor(r, device="cuda")
            zt = torch.zeros_like(rt)
            g.apply_block("precond", rt, zt)
            assert rel(zt.cpu().numpy(), o.P(r)) <= 1e-11
        x = torch.zeros_like(b)
        st = g.solve(b, x, 1e-8)
        g.close()
        xc = x.cpu().numpy()
        assert st.status == 0
        assert np.linalg.norm(s.rhs - s.scipy() @ xc) / np.linalg.norm(s.rhs) <= 1e-8 * 1.001
        if prec == "fp64":
            assert abs(st.iters - ref.iters) <= 1 and rel(xc, ref.x) <= 1e-8, (st.iters, ref.iters)


def _read_oracle_samples(workload):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", f"oracle_{workload}_samples.txt")
    head, idx, val = {}, [], []
    for line in open(path):
        if line.startswith("#"):
            parts = line[1:].split()
            if len(parts) == 2:
                head[parts[0]] = float(parts[1])
            continue
        i, v = line.split()
        idx.append(int(i))
        val.append(float(v))
    return head, np.array(idx), np.array(val)


def test_2d_large_fp64_matches_sampled_oracle(torch_cuda):
    """The 8.9M-DOF Jacobian (1024x512): the FP64 GPU solve against the FP64 oracle's
    own full solve of it, stored at 4000 seeded indices with the solution's 2-norm by
    tests/golden/make_oracle_samples.py (the oracle takes minutes at this size; AMG
    coarse size 500, passed here too): iteration count within +-1, sampled entries and
    the 2-norm within 1e-8."""
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    head, idx, ref = _read_oracle_samples("2d_large")
    s = fsigen.make_system("2d_large")
    assert s.n == int(head["n"])
    g = P.FSISolver.from_system(s, params=P.default_params(2, mass_ratio=8.0, flags=P.FSI_USE_GRAPHS, coarse_max=500))
    g.precond_build("fp64")
    b = torch.tensor(s.rhs, device="cuda")
    x = torch.zeros_like(b)
    st = g.solve(b, x, 1e-8)
    g.close()
    xc = x.cpu().numpy()
    e = rel(xc[idx], ref)
    print(f"[parity] 2d_large: GPU FP64 {st.iters} it, oracle {int(head['iters'])} it, sampled rel. difference "
          f"{e:.3e}, norm {abs(np.linalg.norm(xc) - head['norm2']) / head['norm2']:.3e}")
    assert st.status == 0 and abs(st.iters - int(head["iters"])) <= 1
    assert e <= 1e-8
    assert abs(np.linalg.norm(xc) - head["norm2"]) <= 1e-8 * head["norm2"]
