"""Pins of the oracle's learned correction stage (oracle/learned.py) and of the
generator's node map it reads: IEEE bfloat16 rounding, the 3x3 lattice patch
against mesh coordinates, features against a loop over coordinates, the
correction's homogeneity and locality, a closed form for a constant network,
backpropagation against finite differences, AdamW closed forms, and the FGMRES
accept / fallback rule (an exact correction converges in one iteration, a bad
one is never taken)."""
import struct

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import fsigen
from oracle import OracleSolver
from oracle import learned as L


@pytest.fixture(scope="module")
def tiny():
    cfg = fsigen.CONFIGS["2d_tiny"]
    pb = fsigen.get_problem(cfg)
    nd, pt = pb.node_map()
    sysm = fsigen.make_system(cfg)
    return pb, nd, pt, sysm


def random_bits(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(L.N_PARAMS) * scale
    return L.bf16_bits(w)


# ------------------------------------------------------------------ bfloat16
def test_bf16_rounding_ieee():
    one = 1.0
    cases = {one: 0x3F80, one + 2.0 ** -8: 0x3F80,            # tie -> even (down)
             one + 3 * 2.0 ** -8: 0x3F82,                      # tie -> even (up)
             one + 2.0 ** -8 + 2.0 ** -20: 0x3F81,             # above the tie
             -2.5: 0xC020, 0.0: 0x0000, 2.0 ** -126: 0x0080}
    for v, bits in cases.items():
        assert int(L.bf16_bits(np.float32(v))) == bits, v
    reps = np.array([1.0, -3.5, 0.15625, 2.0 ** 20, -(2.0 ** -10)], np.float64)
    assert np.array_equal(L.bf16_value(L.bf16_bits(reps)), reps)


def test_weights_file_format(tmp_path):
    rng = np.random.default_rng(1)
    bits = rng.integers(0, 0x7F00, L.N_PARAMS).astype(np.uint16)
    si = np.array([1.5, 2, 3, 4, 5], np.float32)
    so = np.array([0.5, 0.25, 8, 16, 32], np.float32)
    path = tmp_path / "w.bin"
    with open(path, "wb") as f:
        f.write(b"FSIMLP01" + struct.pack("<4i", 53, 64, 5, 0) + si.tobytes() + so.tobytes() + bits.tobytes())
    b2, s_in, s_out = L.read_weights(str(path))
    assert np.array_equal(b2, bits) and np.array_equal(s_in, si) and np.array_equal(s_out, so)


# ------------------------------------------------------------------ node map
def test_node_map_matches_coordinates(tiny):
    pb, nd, pt, _ = tiny
    h = np.array(pb.cfg.L[:2]) / np.array(pb.cfg.n) / 2.0      # Q2 lattice spacing
    X = pb.coords
    for a in range(nd.shape[0]):
        v0, u0, p, fl = nd[a]
        assert pb.field[v0] == 0 and pb.comp[v0] == 0 and pb.field[v0 + 1] == 0 and pb.comp[v0 + 1] == 1
        assert pb.field[u0] == 1 and pb.comp[u0] == 0
        assert np.allclose(X[v0], X[u0]) and np.allclose(X[v0], X[v0 + 1])
        ij = np.rint(X[v0] / h).astype(int)
        assert bool(fl & L.FLAG_IODD) == bool(ij[0] % 2) and bool(fl & L.FLAG_JODD) == bool(ij[1] % 2)
        if p >= 0:
            assert pb.field[p] == 2 and np.allclose(X[p], X[v0]) and ij[0] % 2 == 0 and ij[1] % 2 == 0
            assert bool(fl & L.FLAG_PFIX) == bool(pb.fixed[p])
        assert bool(fl & L.FLAG_VFIX) == bool(pb.fixed[v0]) and bool(fl & L.FLAG_UFIX) == bool(pb.fixed[u0])
        for s in range(9):
            di, dj = s % 3 - 1, s // 3 - 1
            q = pt[a, s]
            want = ij + np.array([di, dj])
            inside = 0 <= want[0] <= 2 * pb.cfg.n[0] and 0 <= want[1] <= 2 * pb.cfg.n[1]
            assert (q >= 0) == inside
            if q >= 0:
                assert np.allclose(X[nd[q, 0]], want * h)
    # every DOF belongs to exactly one node
    D = L.node_dofs(nd)
    owned = D[D >= 0]
    assert np.array_equal(np.sort(owned), np.arange(pb.n))


# ------------------------------------------------------------------ features / correction
def test_features_by_coordinate_loop(tiny):
    pb, nd, pt, sysm = tiny
    rng = np.random.default_rng(3)
    rp = rng.standard_normal(pb.n)
    sig = np.array([0.5, 2.0, 3.0, 0.25, 4.0])
    F, rho = L.features(rp, nd, pt, sysm.offsets, sig)
    h = np.array(pb.cfg.L[:2]) / np.array(pb.cfg.n) / 2.0
    cls = L.dof_class(np.arange(pb.n), sysm.offsets)
    by_key = {}
    for d in range(pb.n):
        key = (int(pb.field[d]), int(pb.comp[d])) + tuple(np.rint(pb.coords[d] / h).astype(int))
        by_key[key] = d
    for a in rng.choice(nd.shape[0], 40, replace=False):
        ij = np.rint(pb.coords[nd[a, 0]] / h).astype(int)
        x = []
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                for f, c in ((0, 0), (0, 1), (1, 0), (1, 1), (2, 0)):
                    d = by_key.get((f, c, ij[0] + di, ij[1] + dj))
                    x.append(0.0 if d is None else rp[d] / sig[cls[d]])
        x = np.array(x)
        r = np.sqrt(np.mean(x * x))
        assert rho[a] == pytest.approx(r, rel=1e-13)
        assert np.allclose(F[a, :45], x / r, rtol=1e-12, atol=1e-14)
        par = (ij[0] % 2) + 2 * (ij[1] % 2)
        assert F[a, 45 + par] == 1.0 and F[a, 45:49].sum() == 1.0


def test_correction_homogeneous_and_local(tiny):
    pb, nd, pt, sysm = tiny
    bits = random_bits(5)
    si, so = np.ones(5), np.full(5, 0.5)
    rng = np.random.default_rng(7)
    rp = rng.standard_normal(pb.n)
    rp[pb.fixed] = 0.0
    c = L.correction(rp, nd, pt, sysm.offsets, bits, si, so)
    assert np.allclose(L.correction(2.5 * rp, nd, pt, sysm.offsets, bits, si, so), 2.5 * c, rtol=1e-12, atol=1e-15)
    assert np.all(c[pb.fixed] == 0.0)
    # perturb one DOF of node q: only nodes whose patch holds q may change
    D = L.node_dofs(nd)
    q = int(nd.shape[0] // 2 + 7)
    rp2 = rp.copy()
    rp2[D[q, 0]] += 1.0
    c2 = L.correction(rp2, nd, pt, sysm.offsets, bits, si, so)
    touched = np.unique(np.nonzero(pt == q)[0])
    allowed = np.zeros(pb.n, bool)
    for a in touched:
        allowed[D[a][D[a] >= 0]] = True
    changed = c2 != c
    assert changed.any() and not np.any(changed & ~allowed)


def test_constant_network_closed_form(tiny):
    pb, nd, pt, sysm = tiny
    P = {name: np.zeros(shape) for name, shape in L.SHAPES}
    P["b3"] = np.array([0.5, -1.0, 2.0, 0.25, -4.0])       # bfloat16-exact values
    bits = L.bf16_bits(L.flatten(P))
    si = np.array([1.0, 2.0, 4.0, 0.5, 8.0])
    so = np.array([3.0, 0.5, 0.25, 2.0, 1.0])
    rng = np.random.default_rng(11)
    rp = rng.standard_normal(pb.n)
    c = L.correction(rp, nd, pt, sysm.offsets, bits, si, so)
    _, rho = L.features(rp, nd, pt, sysm.offsets, si)
    D = L.node_dofs(nd)
    M = L.output_mask(nd)
    cls = L.dof_class(np.arange(pb.n), sysm.offsets)
    for a in range(nd.shape[0]):
        for k in range(5):
            d = D[a, k]
            if d < 0:
                continue
            want = P["b3"][k] * rho[a] * so[cls[d]] if M[a, k] else 0.0
            assert c[d] == pytest.approx(want, rel=1e-14, abs=0.0)


# ------------------------------------------------------------------ training
def test_residual_gradient_finite_differences(tiny):
    pb, nd, pt, sysm = tiny
    A = sp.csr_matrix((sysm.vals, sysm.colind, sysm.rowptr), shape=(pb.n, pb.n))
    rng = np.random.default_rng(13)
    rp = rng.standard_normal(pb.n)
    rp[pb.fixed] = 0.0
    params = rng.standard_normal(L.N_PARAMS) * 0.2
    si = np.array([1.0, 1.0, 1e-3, 1.0, 1.0])
    so = np.array([1e-3, 1e-3, 1e-5, 1e-3, 1e-2])
    loss, g = L.residual_loss_and_grad(params, rp, A, nd, pt, sysm.offsets, si, so)
    assert loss > 0
    offs = {}
    k = 0
    for name, shape in L.SHAPES:
        offs[name] = (k, int(np.prod(shape)))
        k += int(np.prod(shape))
    idx = [offs[nm][0] + int(rng.integers(0, offs[nm][1])) for nm in offs for _ in range(4)]
    for i in idx:
        eps = 1e-6 * max(1.0, abs(params[i]))
        p1, p2 = params.copy(), params.copy()
        p1[i] += eps
        p2[i] -= eps
        l1, _ = L.residual_loss_and_grad(p1, rp, A, nd, pt, sysm.offsets, si, so)
        l2, _ = L.residual_loss_and_grad(p2, rp, A, nd, pt, sysm.offsets, si, so)
        fd = (l1 - l2) / (2 * eps)
        assert g[i] == pytest.approx(fd, rel=2e-5, abs=1e-9 * max(1.0, np.abs(g).max())), i


def test_adamw_closed_forms():
    rng = np.random.default_rng(17)
    w0 = rng.standard_normal(50)
    g = rng.standard_normal(50)
    z = np.zeros(50)
    # bias-corrected first step moves each weight by lr against the gradient's sign
    w1, m, v = L.adamw_step(w0, g, z, z, 1, lr=0.01, eps=0.0)
    assert np.allclose(w1, w0 - 0.01 * np.sign(g), rtol=0, atol=1e-15)
    # with a constant gradient every step has the same length lr
    w = w0.copy()
    m, v = z.copy(), z.copy()
    for t in range(1, 8):
        w_next, m, v = L.adamw_step(w, g, m, v, t, lr=0.01, eps=0.0)
        assert np.allclose(w_next - w, -0.01 * np.sign(g), rtol=0, atol=1e-14)
        w = w_next
    # decoupled weight decay acts alone when the gradient is zero
    w2, _, _ = L.adamw_step(w0, np.zeros(50), z, z, 1, lr=0.1, eps=1e-8, weight_decay=0.5)
    assert np.allclose(w2, w0 * (1 - 0.05), rtol=1e-15)


# ------------------------------------------------------------------ FGMRES accept rule
def test_exact_correction_converges_in_one_iteration(tiny):
    pb, nd, pt, sysm = tiny
    A = sp.csr_matrix((sysm.vals, sysm.colind, sysm.rowptr), shape=(pb.n, pb.n)).tocsc()
    lu = spla.splu(A)
    S = OracleSolver.from_system(sysm)
    res = S.solve(sysm.rhs, 1e-10, correct=lambda r: lu.solve(r))
    assert res.converged and res.iters == 1 and res.accepted == 1


def test_bad_correction_is_never_taken(tiny):
    pb, nd, pt, sysm = tiny
    A = sp.csr_matrix((sysm.vals, sysm.colind, sysm.rowptr), shape=(pb.n, pb.n)).tocsc()
    lu = spla.splu(A)
    S = OracleSolver.from_system(sysm)
    plain = S.solve(sysm.rhs, 1e-8)
    bad = S.solve(sysm.rhs, 1e-8, correct=lambda r: -3.0 * lu.solve(r))   # ||r' - A c|| = 4 ||r'||
    assert bad.accepted == 0
    assert bad.iters == plain.iters and np.array_equal(bad.x, plain.x) and bad.history == plain.history
