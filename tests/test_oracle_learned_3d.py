"""Pins of the learned stage in 3D (oracle/learned.py and the generator's node map):
the 3x3x3 lattice patch and the flags against mesh coordinates, the 201 features
against a loop over coordinates, homogeneity and locality of the correction, a
constant network in closed form, and backpropagation against finite differences."""
import numpy as np
import pytest
import scipy.sparse as sp

import fsigen
from oracle import learned as L


@pytest.fixture(scope="module")
def tiny3():
    cfg = fsigen.CONFIGS["3d"].with_(name="3d_4x2x2", n=(4, 2, 2))
    pb = fsigen.get_problem(cfg)
    nd, pt = pb.node_map()
    sysm = fsigen.make_system(cfg)
    return pb, nd, pt, sysm


def random_bits3(seed, scale=0.2):
    return L.bf16_bits(np.random.default_rng(seed).standard_normal(L.N_PARAMS_3D) * scale)


def lattice(pb):
    h = np.array(pb.cfg.L[:3]) / np.array(pb.cfg.n) / 2.0
    return h, {k: d for d, k in enumerate(
        (int(pb.field[d]), int(pb.comp[d])) + tuple(np.rint(pb.coords[d] / h).astype(int)) for d in range(pb.n))}


def test_layout_3d():
    assert L.layout(3) == (201, 7, 189, 27, 7, 8) and L.layout(2) == (53, 5, 45, 9, 5, 4)
    assert L.N_PARAMS_3D == 201 * 64 + 64 + 64 * 64 + 64 + 64 * 7 + 7


def test_node_map_3d_matches_coordinates(tiny3):
    pb, nd, pt, _ = tiny3
    assert pt.shape == (nd.shape[0], 27)
    h = np.array(pb.cfg.L[:3]) / np.array(pb.cfg.n) / 2.0
    X = pb.coords
    n2 = 2 * np.array(pb.cfg.n)
    for a in range(nd.shape[0]):
        v0, u0, p, fl = nd[a]
        for i in range(3):
            assert pb.field[v0 + i] == 0 and pb.comp[v0 + i] == i and pb.field[u0 + i] == 1 and pb.comp[u0 + i] == i
        ijk = np.rint(X[v0] / h).astype(int)
        assert np.allclose(X[u0], X[v0])
        assert bool(fl & L.FLAG_IODD) == bool(ijk[0] % 2) and bool(fl & L.FLAG_JODD) == bool(ijk[1] % 2)
        assert bool(fl & L.FLAG_KODD) == bool(ijk[2] % 2)
        if p >= 0:
            assert pb.field[p] == 2 and np.allclose(X[p], X[v0]) and not np.any(ijk % 2)
            assert bool(fl & L.FLAG_PFIX) == bool(pb.fixed[p])
        else:
            assert np.any(ijk % 2)
        assert bool(fl & L.FLAG_VFIX) == bool(pb.fixed[v0]) and bool(fl & L.FLAG_UFIX) == bool(pb.fixed[u0])
        for s in range(27):
            d = np.array([s % 3 - 1, (s // 3) % 3 - 1, s // 9 - 1])
            want = ijk + d
            inside = np.all(want >= 0) and np.all(want <= n2)
            q = pt[a, s]
            assert (q >= 0) == inside
            if q >= 0:
                assert np.allclose(X[nd[q, 0]], want * h)
    D = L.node_dofs(nd, 3)
    owned = D[D >= 0]
    assert np.array_equal(np.sort(owned), np.arange(pb.n))


def test_features_3d_by_coordinate_loop(tiny3):
    pb, nd, pt, sysm = tiny3
    rng = np.random.default_rng(31)
    rp = rng.standard_normal(pb.n)
    sig = np.array([0.5, 2.0, 3.0, 0.25, 4.0])
    F, rho = L.features(rp, nd, pt, sysm.offsets, sig)
    assert F.shape == (nd.shape[0], 201)
    h, by_key = lattice(pb)
    cls = L.dof_class(np.arange(pb.n), sysm.offsets)
    comps = [(0, 0), (0, 1), (0, 2), (1, 0), (1, 1), (1, 2), (2, 0)]
    for a in rng.choice(nd.shape[0], 30, replace=False):
        ijk = np.rint(pb.coords[nd[a, 0]] / h).astype(int)
        x = []
        for dk in (-1, 0, 1):
            for dj in (-1, 0, 1):
                for di in (-1, 0, 1):
                    for f, c in comps:
                        d = by_key.get((f, c, ijk[0] + di, ijk[1] + dj, ijk[2] + dk))
                        x.append(0.0 if d is None else rp[d] / sig[cls[d]])
        x = np.array(x)
        r = np.sqrt(np.mean(x * x))
        assert rho[a] == pytest.approx(r, rel=1e-13)
        assert np.allclose(F[a, :189], x / r, rtol=1e-12, atol=1e-14)
        par = (ijk[0] % 2) + 2 * (ijk[1] % 2) + 4 * (ijk[2] % 2)
        assert F[a, 189 + par] == 1.0 and F[a, 189:197].sum() == 1.0
        fl = nd[a, 3]
        for k, bit in enumerate((L.FLAG_SOLID, L.FLAG_VFIX, L.FLAG_UFIX, L.FLAG_IFACE)):
            assert F[a, 197 + k] == float(bool(fl & bit))


def test_correction_3d_homogeneous_and_local(tiny3):
    pb, nd, pt, sysm = tiny3
    bits = random_bits3(5)
    si, so = np.ones(5), np.full(5, 0.5)
    rng = np.random.default_rng(37)
    rp = rng.standard_normal(pb.n)
    rp[pb.fixed] = 0.0
    c = L.correction(rp, nd, pt, sysm.offsets, bits, si, so)
    assert np.allclose(L.correction(2.5 * rp, nd, pt, sysm.offsets, bits, si, so), 2.5 * c, rtol=1e-12, atol=1e-15)
    assert np.all(c[pb.fixed] == 0.0) and np.any(c != 0.0)
    D = L.node_dofs(nd, 3)
    q = int(nd.shape[0] // 2)
    rp2 = rp.copy()
    rp2[D[q, 0] + 2] += 1.0          # the z velocity of node q
    c2 = L.correction(rp2, nd, pt, sysm.offsets, bits, si, so)
    allowed = np.zeros(pb.n, bool)
    for a in np.unique(np.nonzero(pt == q)[0]):
        allowed[D[a][D[a] >= 0]] = True
    changed = c2 != c
    assert changed.any() and not np.any(changed & ~allowed)


def test_constant_network_3d_closed_form(tiny3):
    pb, nd, pt, sysm = tiny3
    P = {name: np.zeros(shape) for name, shape in L.shapes(3)}
    P["b3"] = np.array([0.5, -1.0, 2.0, 0.25, -4.0, 1.5, -0.75])     # bfloat16-exact values
    bits = L.bf16_bits(L.flatten(P))
    si = np.array([1.0, 2.0, 4.0, 0.5, 8.0])
    so = np.array([3.0, 0.5, 0.25, 2.0, 1.0])
    rp = np.random.default_rng(41).standard_normal(pb.n)
    c = L.correction(rp, nd, pt, sysm.offsets, bits, si, so)
    _, rho = L.features(rp, nd, pt, sysm.offsets, si)
    D, M = L.node_dofs(nd, 3), L.output_mask(nd, 3)
    cls = L.dof_class(np.arange(pb.n), sysm.offsets)
    for a in range(nd.shape[0]):
        for k in range(7):
            d = D[a, k]
            if d >= 0:
                want = P["b3"][k] * rho[a] * so[cls[d]] if M[a, k] else 0.0
                assert c[d] == pytest.approx(want, rel=1e-14, abs=0.0)


def test_residual_gradient_3d_finite_differences(tiny3):
    pb, nd, pt, sysm = tiny3
    A = sp.csr_matrix((sysm.vals, sysm.colind, sysm.rowptr), shape=(pb.n, pb.n))
    rng = np.random.default_rng(43)
    rp = rng.standard_normal(pb.n)
    rp[pb.fixed] = 0.0
    params = rng.standard_normal(L.N_PARAMS_3D) * 0.1
    si = np.array([1.0, 1.0, 1e-3, 1.0, 1.0])
    so = np.array([1e-3, 1e-3, 1e-5, 1e-3, 1e-2])
    loss, g = L.residual_loss_and_grad(params, rp, A, nd, pt, sysm.offsets, si, so)
    assert loss > 0 and g.shape == (L.N_PARAMS_3D,)
    offs, k = {}, 0
    for name, shape in L.shapes(3):
        offs[name] = (k, int(np.prod(shape)))
        k += int(np.prod(shape))
    idx = [offs[nm][0] + int(rng.integers(0, offs[nm][1])) for nm in offs for _ in range(3)]
    for i in idx:
        eps = 1e-6 * max(1.0, abs(params[i]))
        p1, p2 = params.copy(), params.copy()
        p1[i] += eps
        p2[i] -= eps
        l1, _ = L.residual_loss_and_grad(p1, rp, A, nd, pt, sysm.offsets, si, so)
        l2, _ = L.residual_loss_and_grad(p2, rp, A, nd, pt, sysm.offsets, si, so)
        fd = (l1 - l2) / (2 * eps)
        assert g[i] == pytest.approx(fd, rel=2e-5, abs=1e-9 * max(1.0, np.abs(g).max())), i
