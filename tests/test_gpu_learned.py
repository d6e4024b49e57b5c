"""Parity of the learned correction stage's CUDA kernels (through the C ABI) with
the FP64 oracle (oracle/learned.py): features, the MLP correction, the FGMRES
accept / fallback rule inside whole solves, the residual harvest, the training
gradient and the AdamW step.

Tolerances (FP32 kernels against FP64 arithmetic on the same bfloat16 weights):
features are r'/sigma in FP32 divided by an FP32 RMS, within 2e-6 relative of
their O(1) size; the MLP accumulates at most 64 FP32 products per unit through
three layers, so corrections agree to 5e-5 of each class's largest entry;
gradients additionally sum per-node products over all nodes (FP32 within a
block, FP64 across blocks): 5e-4 of the largest entry.  Solves with the stage
reach the 1e-8 relative residual with iterations and accepted corrections within
+-1 of the oracle's (a decision can only flip at a near-tie of the two residual
norms); the FP32 MLP steers another Krylov trajectory than the FP64 oracle's,
so, like the FP32-AMG form, the solution is measured against the manufactured x*:
within 10x of the FP64 oracle's own error (1e-6 when that is smaller)."""
import numpy as np
import pytest
import scipy.sparse as sp

import fsigen
import oracle
from oracle import learned as L

pytestmark = pytest.mark.gpu

CASES = {
    "2d_16x16": fsigen.CONFIGS["2d_tiny"],
    "2d_37x19_ragged": fsigen.CONFIGS["2d_tiny"].with_(name="2d_37x19", n=(37, 19), state_seed=3, rhs_seed=5),
}


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
        cfg = CASES[name]
        s = fsigen.make_system(cfg)
        pb = fsigen.get_problem(cfg)
        nd, pt = pb.node_map()
        g = P.FSISolver.from_system(s, params=P.default_params(2))
        g.precond_build("fp64")
        g.learned_setup(nd, pt)
        _cache[name] = (s, pb, nd, pt, g)
    return _cache[name]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def random_bits(seed, scale=0.3):
    return L.bf16_bits(np.random.default_rng(seed).standard_normal(L.N_PARAMS) * scale)


def scaled_identity_bits(alpha):
    """A network whose output is y_k = alpha_k x_{centre,k}: both hidden layers
    stay in the linear range of gelu by a bias of 16 (|x| <= sqrt(45)), removed at
    the output.  All values are exact in bfloat16."""
    P = {name: np.zeros(shape) for name, shape in L.SHAPES}
    for k in range(5):
        P["W1"][20 + k, k] = 1.0          # centre slot 4: features 20..24
        P["b1"][k] = 16.0
        P["W2"][k, k] = 1.0
        P["W3"][k, k] = alpha[k]
        P["b3"][k] = -16.0 * alpha[k]
    return L.bf16_bits(L.flatten(P))


def lsq_scales(s):
    """Class scales s_c minimising ||r'_0 - A sum_c s_c E_c r'_0|| (E_c: restriction
    to class c, r'_0 = v_0 - A P^-1 v_0 of the oracle's first FGMRES step): with the
    scaled-identity network (sigma_in = 1, sigma_out = |s_c|) the correction is
    accepted at least in the first iteration, so the accept branch runs."""
    o = oracle.OracleSolver.from_system(s)
    A = s.scipy()
    v0 = s.rhs / np.linalg.norm(s.rhs)
    rp = v0 - A @ o.P(v0)
    cols = []
    for c in range(5):
        e = np.zeros(s.n)
        sl = slice(int(s.offsets[c]), int(s.offsets[c + 1]))
        e[sl] = rp[sl]
        cols.append(A @ e)
    coef, *_ = np.linalg.lstsq(np.stack(cols, 1), rp, rcond=None)
    alpha = np.array([1.0, 1.0, 1.0, 1.0, 1.0 if coef[4] >= 0 else -1.0])
    mag = np.abs(coef)
    mag[:4][coef[:4] < 0] = 0.0                      # v and u outputs keep alpha = +1
    so = np.maximum(mag, 1e-30).astype(np.float32)
    return np.ones(5, np.float32), so, alpha


def richardson_scales(s):
    """sigma_out / sigma_in per class = 1 / mean |diag| of the class rows: the
    scaled-identity network then applies a damped, class-wise Jacobi step."""
    A = s.scipy()
    d = np.abs(A.diagonal())
    off = s.offsets
    si = np.ones(5, np.float32)
    so = np.array([1.0 / max(d[off[c]:off[c + 1]][~s.fixed[off[c]:off[c + 1]]].mean(), 1e-30) for c in range(5)],
                  np.float32)
    return si, so


@pytest.mark.parametrize("name", list(CASES))
def test_features_match_oracle(name, torch_cuda):
    torch = torch_cuda
    s, pb, nd, pt, g = case(name, torch)
    rng = np.random.default_rng(21)
    rp = rng.standard_normal(s.n) * np.exp(rng.uniform(-3, 3, s.n))
    si = np.array([0.5, 2.0, 1e-3, 4.0, 0.25], np.float32)
    g.learned_set_weights(si, np.ones(5, np.float32), random_bits(1))
    F = torch.empty((nd.shape[0], 53), dtype=torch.float32, device="cuda")
    rho = torch.empty(nd.shape[0], dtype=torch.float32, device="cuda")
    g.learned_features(torch.tensor(rp, device="cuda"), F, rho)
    Fo, rho_o = L.features(rp, nd, pt, s.offsets, si.astype(np.float64))
    assert np.allclose(rho.cpu().numpy(), rho_o, rtol=2e-6, atol=0)
    assert np.abs(F.cpu().numpy() - Fo).max() <= 2e-6 * np.sqrt(45)


def check_correction(s, nd, pt, g, torch, rp, si, so, bits):
    c = torch.full((s.n,), np.nan, dtype=torch.float64, device="cuda")
    g.learned_apply(torch.tensor(rp, device="cuda"), c)
    cg = c.cpu().numpy()
    co = L.correction(rp, nd, pt, s.offsets, bits, si.astype(np.float64), so.astype(np.float64))
    assert np.all(np.isfinite(cg)), "every DOF of c must be written"
    assert np.all(cg[s.fixed] == 0.0)
    cls = L.dof_class(np.arange(s.n), s.offsets)
    for k in range(5):
        sel = cls == k
        if sel.any() and np.abs(co[sel]).max() > 0:
            assert np.abs(cg[sel] - co[sel]).max() <= 5e-5 * np.abs(co[sel]).max(), k
    return cg


# the MLP on the tensor cores (tcgen05, the default) and on the CUDA cores
UNITS = {"tensor_cores": 0, "cuda_cores": 256}


@pytest.mark.parametrize("unit", list(UNITS))
@pytest.mark.parametrize("name", list(CASES))
def test_correction_matches_oracle(name, unit, torch_cuda):
    """Several 128-node tiles and a ragged last one (1,089 and 2,925 nodes)."""
    torch = torch_cuda
    s, pb, nd, pt, g = case(name, torch)
    rng = np.random.default_rng(22)
    rp = rng.standard_normal(s.n)
    si = np.array([1.0, 2.0, 0.5, 4.0, 0.25], np.float32)
    so = np.array([3.0, 0.5, 0.25, 2.0, 1.5], np.float32)
    g.set_flags(UNITS[unit])
    try:
        for seed in (2, 3):
            bits = random_bits(seed)
            g.learned_set_weights(si, so, bits)
            check_correction(s, nd, pt, g, torch, rp, si, so, bits)
    finally:
        g.set_flags(0)


def test_correction_2d_256x128_both_units(torch_cuda):
    """131,841 nodes: 1,031 tiles, several per CTA of the tensor-core kernel (its
    barrier phases alternate across tiles); both units against the oracle and
    against each other, with the committed trained weights."""
    torch = torch_cuda
    import os
    import paper_1801_05648_gb300 as P
    cfg = fsigen.CONFIGS["2d_mid"]
    s = fsigen.make_system(cfg)
    nd, pt = fsigen.get_problem(cfg).node_map()
    g = P.FSISolver.from_system(s, params=P.default_params(2))
    try:
        g.learned_setup(nd, pt)
        path = os.path.join(os.path.dirname(P.__file__), "weights", "mlp_fsi2d_256x128.bin")
        bits, si, so = L.read_weights(path)
        g.learned_set_weights(np.asarray(si, np.float32), np.asarray(so, np.float32), bits)
        rp = np.random.default_rng(24).standard_normal(s.n) * np.exp(np.random.default_rng(25).uniform(-2, 2, s.n))
        out = {}
        for unit, fl in UNITS.items():
            g.set_flags(fl)
            out[unit] = check_correction(s, nd, pt, g, torch, rp, np.asarray(si, np.float32),
                                         np.asarray(so, np.float32), bits)
        a, b = out["tensor_cores"], out["cuda_cores"]
        assert np.abs(a - b).max() <= 5e-5 * np.abs(b).max()
    finally:
        g.close()


def test_scaled_identity_network_closed_form(torch_cuda):
    torch = torch_cuda
    s, pb, nd, pt, g = case("2d_37x19_ragged", torch)
    alpha = np.array([0.5, 0.25, 1.0, 2.0, -0.5])
    si = np.array([1.0, 2.0, 0.5, 4.0, 0.25], np.float32)
    so = np.array([3.0, 0.5, 0.25, 2.0, 1.5], np.float32)
    g.learned_set_weights(si, so, scaled_identity_bits(alpha))
    rp = np.random.default_rng(23).standard_normal(s.n)
    c = torch.empty(s.n, dtype=torch.float64, device="cuda")
    g.learned_apply(torch.tensor(rp, device="cuda"), c)
    cls = L.dof_class(np.arange(s.n), s.offsets)
    D = L.node_dofs(nd)
    want = np.zeros(s.n)
    M = L.output_mask(nd)
    for k in range(5):
        ok = (D[:, k] >= 0) & (M[:, k] > 0)
        d = D[ok, k]
        want[d] = alpha[k] * rp[d] / si[cls[d]] * so[cls[d]]
    # the bias shift of 16 costs 16 * 2^-24 of the unit-RMS features in FP32
    scale = np.abs(want).max()
    assert np.abs(c.cpu().numpy() - want).max() <= 1e-5 * scale


@pytest.mark.parametrize("name", list(CASES))
def test_learned_solve_matches_oracle(name, torch_cuda):
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    s, pb, nd, pt, g = case(name, torch)
    si, so, alpha = lsq_scales(s)
    bits = scaled_identity_bits(alpha)
    g.learned_set_weights(si, so, bits)
    o = oracle.OracleSolver.from_system(s)
    err64 = rel(o.solve(s.rhs, 1e-8).x, s.x_exact)
    stage = L.LearnedStage(nd, pt, s.offsets, bits, si.astype(np.float64), so.astype(np.float64))
    b = torch.tensor(s.rhs, device="cuda")
    for tau in (1.0, 0.9):
        ref = o.solve(s.rhs, 1e-8, correct=stage, accept=tau)
        g.set_learned_accept(tau)
        for flags in (0, P.FSI_USE_GRAPHS):
            g.set_flags(flags | P.FSI_LEARNED)
            x = torch.zeros_like(b)
            st = g.solve(b, x, 1e-8)
            xc = x.cpu().numpy()
            assert st.status == 0 and st.true_relres <= 1e-8
            assert np.linalg.norm(s.rhs - s.scipy() @ xc) / np.linalg.norm(s.rhs) <= 1e-8 * 1.001
            assert abs(st.iters - ref.iters) <= 1, (tau, st.iters, ref.iters)
            assert abs(st.learned_accepted - ref.accepted) <= 1, (tau, st.learned_accepted, ref.accepted)
            # the FP32 MLP steers another Krylov trajectory than the FP64 oracle's:
            # measured like the FP32-AMG form, against x*
            assert rel(xc, s.x_exact) <= max(10.0 * err64, 1e-6), (rel(xc, s.x_exact), err64)
        if tau == 1.0:
            assert ref.accepted >= 1          # the accept branch ran
    g.set_learned_accept(0.1)
    g.set_flags(0)


def test_bad_correction_falls_back_bit_identically(torch_cuda):
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    s, pb, nd, pt, g = case("2d_16x16", torch)
    P_ = {name: np.zeros(shape) for name, shape in L.SHAPES}
    P_["b3"][:] = 1.0e4                        # c = 1e4 rho sigma_out: ||r' - A c|| >> ||r'||
    g.learned_set_weights(np.ones(5, np.float32), np.ones(5, np.float32), L.bf16_bits(L.flatten(P_)))
    b = torch.tensor(s.rhs, device="cuda")
    for flags in (0, P.FSI_USE_GRAPHS):
        g.set_flags(flags)
        x0 = torch.zeros_like(b)
        plain = g.solve(b, x0, 1e-8)
        g.set_flags(flags | P.FSI_LEARNED)
        x1 = torch.zeros_like(b)
        lst = g.solve(b, x1, 1e-8)
        assert lst.learned_accepted == 0
        assert lst.iters == plain.iters and lst.history == plain.history
        assert torch.equal(x0, x1)
    g.set_flags(0)


def test_learned_graph_replay_is_bit_identical(torch_cuda):
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    s, pb, nd, pt, g = case("2d_37x19_ragged", torch)
    si, so = richardson_scales(s)
    g.learned_set_weights(si, so, scaled_identity_bits(np.full(5, 0.5)))
    b = torch.tensor(s.rhs, device="cuda")
    xs = []
    for flags in (P.FSI_LEARNED, P.FSI_LEARNED | P.FSI_USE_GRAPHS):
        g.set_flags(flags)
        x = torch.zeros_like(b)
        st = g.solve(b, x, 1e-8)
        xs.append((x, st.iters, st.learned_accepted))
    assert torch.equal(xs[0][0], xs[1][0]) and xs[0][1:] == xs[1][1:]
    g.set_flags(0)


def test_harvest_first_residual(torch_cuda):
    torch = torch_cuda
    s, pb, nd, pt, g = case("2d_16x16", torch)
    b = torch.tensor(s.rhs, device="cuda")
    buf = torch.zeros((4, s.n), dtype=torch.float64, device="cuda")
    g.set_harvest(buf, 4)
    x = torch.zeros_like(b)
    st = g.solve(b, x, 1e-8)
    g.set_harvest(None)
    assert st.iters >= 4
    v0 = b / torch.linalg.vector_norm(b)
    z = torch.empty_like(b)
    g.apply_block("precond", v0, z)
    w = torch.empty_like(b)
    g.apply_operator(z, w)
    want = (v0 - w).cpu().numpy()
    got = buf[0].cpu().numpy()
    # r' = v - A P^-1 v cancels (||r'|| ~ 3e-4 here): rounding is relative to ||v|| = 1
    assert np.linalg.norm(got - want) <= 1e-13
    # later vectors: orthonormal Krylov basis vectors minus A P^-1 of them, all non-zero
    assert all(float(torch.linalg.vector_norm(buf[j])) > 0 for j in range(4))


def test_trainer_gradient_and_adamw_match_oracle(torch_cuda):
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    s, pb, nd, pt, g = case("2d_37x19_ragged", torch)
    rng = np.random.default_rng(31)
    rp = rng.standard_normal(s.n)
    rp[s.fixed] = 0.0
    si = np.array([1.0, 0.5, 1e-3, 2.0, 0.5], np.float32)
    so = np.array([1e-3, 1e-3, 1e-5, 1e-3, 1e-2], np.float32)
    tr = P.Trainer(lr=1e-2, seed=4, sigma_in=list(si), sigma_out=list(so))
    w = (rng.standard_normal(L.N_PARAMS) * 0.2).astype(np.float32)
    tr.set_master(w)
    m0, bits, g0 = tr.get()
    assert np.array_equal(m0, w) and np.array_equal(bits, L.bf16_bits(w)) and not g0.any()
    r = torch.tensor(rp, device="cuda")
    loss = tr.step(g, r)
    loss_o, grad_o = L.residual_loss_and_grad(L.bf16_value(bits), rp, s.scipy(), nd, pt, s.offsets,
                                              si.astype(np.float64), so.astype(np.float64))
    assert loss == pytest.approx(loss_o, rel=1e-5)
    assert tr.loss(g, r) == pytest.approx(loss, rel=1e-12)
    _, _, grad = tr.get()
    assert np.abs(grad - grad_o).max() <= 5e-4 * np.abs(grad_o).max()
    # one AdamW step from zero moments with the GPU's own gradient
    tr.update(g, 1e-2)
    m1, bits1, g1 = tr.get()
    w_o, _, _ = L.adamw_step(w.astype(np.float64), grad.astype(np.float64), np.zeros(L.N_PARAMS),
                             np.zeros(L.N_PARAMS), 1, lr=1e-2, eps=1e-8)
    assert np.abs(m1 - w_o).max() <= 1e-6 * max(1.0, np.abs(w_o).max())
    assert np.array_equal(bits1, L.bf16_bits(m1)) and not g1.any()


def test_training_lowers_the_loss(torch_cuda, tmp_path):
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    s, pb, nd, pt, g = case("2d_16x16", torch)
    b = torch.tensor(s.rhs, device="cuda")
    buf = torch.zeros((6, s.n), dtype=torch.float64, device="cuda")
    g.set_harvest(buf, 6)
    g.solve(b, torch.zeros_like(b), 1e-8)
    g.set_harvest(None)
    si, so = richardson_scales(s)
    tr = P.Trainer(lr=3e-3, seed=0, sigma_in=list(si), sigma_out=list(so))
    first = np.mean([tr.loss(g, buf[j]) for j in range(6)])
    for _ in range(60):
        for j in range(6):
            tr.step(g, buf[j])
        tr.update(g)
    last = np.mean([tr.loss(g, buf[j]) for j in range(6)])
    assert last < first
    # the saved file reproduces the trainer's weights in the solver
    path = tmp_path / "w.bin"
    tr.save(str(path))
    bits_f, si_f, so_f = L.read_weights(str(path))
    _, bits_t, _ = tr.get()
    assert np.array_equal(bits_f, bits_t) and np.allclose(si_f, si) and np.allclose(so_f, so)
    g.learned_load(str(path))
    c1 = torch.empty_like(b)
    g.learned_apply(buf[0], c1)
    g.learned_set_weights(si, so, bits_t)
    c2 = torch.empty_like(b)
    g.learned_apply(buf[0], c2)
    assert torch.equal(c1, c2)


def test_learned_stage_argument_errors(torch_cuda):
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    s, pb, nd, pt, g = case("2d_16x16", torch)
    bad = nd.copy()
    bad[1, 0] = bad[0, 0]                       # a DOF owned by two nodes
    with pytest.raises(P.FSIError) as e:
        g.learned_setup(bad, pt)
    assert e.value.code == -1
    badp = pt.copy()
    badp[0, 0] = nd.shape[0]                    # patch entry out of range
    with pytest.raises(P.FSIError):
        g.learned_setup(nd, badp)
    with pytest.raises(P.FSIError):
        g.learned_set_weights(np.zeros(5, np.float32), np.ones(5, np.float32), random_bits(0))
    with pytest.raises(P.FSIError):
        g.set_flags(P.FSI_CLUSTER_COARSE)
    g.learned_setup(nd, pt)                     # the context stays usable
