"""The C-ABI library builds, loads and exports every symbol include/fsi.h
declares; argument validation rejects malformed input before touching the
device (so these run without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1801_05648_gb300 import build
    build.build()
    import paper_1801_05648_gb300 as P
    return P.load_library()


def header_functions():
    text = open(os.path.join(ROOT, "include", "fsi.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fsi_[a-z_]+)\s*\(", text)))


def test_header_symbols_exported(lib):
    names = header_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    import paper_1801_05648_gb300 as P
    assert sorted(P.EXPORTED) == names


def test_peaks_library_exports_its_header(lib):
    """libfsi_peaks.so (the FMA-throughput probes of the rooflines) loads and exports
    every function include/fsi_peaks.h declares."""
    import paper_1801_05648_gb300 as P
    text = open(os.path.join(ROOT, "include", "fsi_peaks.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = sorted(set(re.findall(r"\b(fsi_[a-z_]+)\s*\(", text)))
    assert names == sorted(P.fsi.PEAKS_EXPORTED)
    peaks = ctypes.CDLL(P.fsi.PEAKS_LIB_PATH)
    for name in names:
        assert hasattr(peaks, name), name
    # argument validation needs no device
    f = peaks.fsi_probe_fma_rate
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                  ctypes.POINTER(ctypes.c_double)]
    out = ctypes.c_double()
    assert f(16, 10, 1, ctypes.byref(out), None) == -1
    assert f(64, 0, 1, ctypes.byref(out), None) == -1
    assert f(64, 10, 1, None, None) == -1


def test_default_params(lib):
    import paper_1801_05648_gb300 as P
    p2, p3 = P.default_params(2), P.default_params(3)
    assert (p2.restart, p2.maxit, p2.cheb_degree, p2.vcycles_solid, p2.mass_degree) == (100, 1000, 4, 2, 12)
    assert p2.mass_ratio == 8.0 and p3.mass_ratio == 20.0
    assert p2.strength_theta == 0.08 and p2.dt_theta == 0.01
    import oracle
    assert p2.coarse_max == oracle.AMGParams().coarse_max == 1500     # the oracle's default is the library's
    assert (p2.cheb_degree_coarse, p2.spmv_prefetch, p2.cluster_max_bytes) == (2, 1, 6.0e6)
    assert p2.fluid_gmres_iters == 4 and P.FSI_FLUID_GMRES == 128 and P.FSI_MLP_CUDA_CORES == 256
    assert p2.precond_variant == P.FSI_PRECOND_LDU == 0 and p2.spmv_lane_shift == 0 and p2.spmv_stage == 0


def _setup(lib, dim, n, rowptr, colind, vals, off, params=None):
    import paper_1801_05648_gb300 as P
    h = ctypes.c_void_p()
    ip = lambda a, t: a.ctypes.data_as(ctypes.POINTER(t))
    rc = lib.fsi_setup(ctypes.byref(h), dim, n, ip(rowptr, ctypes.c_int64), ip(colind, ctypes.c_int32),
                       ip(vals, ctypes.c_double), ip(off, ctypes.c_int64), None,
                       None if params is None else ctypes.byref(params), None)
    return rc, h, lib.fsi_last_error(None).decode()


def _tiny_csr():
    # 4x4 identity-like system, offsets: m=2 | s_v=0 | s_u=0 | f_v=0 | p=2 (dim 2)
    rowptr = np.array([0, 1, 2, 3, 4], np.int64)
    colind = np.array([0, 1, 2, 3], np.int32)
    vals = np.ones(4)
    off = np.array([0, 2, 2, 2, 2, 4], np.int64)
    return rowptr, colind, vals, off


def test_rejects_unsorted_columns(lib):
    rp = np.array([0, 2, 3, 4, 5], np.int64)
    ci = np.array([1, 0, 1, 2, 3], np.int32)
    rc, h, msg = _setup(lib, 2, 4, rp, ci, np.ones(5), np.array([0, 2, 2, 2, 2, 4], np.int64))
    assert rc == -1 and "increasing" in msg and not h.value


def test_rejects_out_of_range_and_nonfinite(lib):
    rp, ci, va, off = _tiny_csr()
    bad = ci.copy(); bad[2] = 7
    rc, h, msg = _setup(lib, 2, 4, rp, bad, va, off)
    assert rc == -1 and "range" in msg
    nan = va.copy(); nan[1] = np.nan
    rc, h, msg = _setup(lib, 2, 4, rp, ci, nan, off)
    assert rc == -1 and "finite" in msg


def test_rejects_bad_offsets_and_dim(lib):
    rp, ci, va, off = _tiny_csr()
    rc, _, msg = _setup(lib, 2, 4, rp, ci, va, np.array([0, 3, 3, 3, 3, 4], np.int64))
    assert rc == -1 and "multiples" in msg
    rc, _, msg = _setup(lib, 4, 4, rp, ci, va, off)
    assert rc == -1 and "dim" in msg
    rc, _, msg = _setup(lib, 2, 4, rp, ci, va, np.array([0, 2, 2, 2, 2, 5], np.int64))
    assert rc == -1


def test_rejects_bad_params(lib):
    import paper_1801_05648_gb300 as P
    rp, ci, va, off = _tiny_csr()
    p = P.default_params(2, restart=0)
    rc, _, msg = _setup(lib, 2, 4, rp, ci, va, off, p)
    assert rc == -1 and "restart" in msg
    for k in (0, 33):
        rc, _, msg = _setup(lib, 2, 4, rp, ci, va, off, P.default_params(2, fluid_gmres_iters=k))
        assert rc == -1 and "fluid_gmres_iters" in msg
    rc, _, msg = _setup(lib, 2, 4, rp, ci, va, off, P.default_params(2, flags=512))
    assert rc == -1 and "flag" in msg
    for v in (-1, 4):
        rc, _, msg = _setup(lib, 2, 4, rp, ci, va, off, P.default_params(2, precond_variant=v))
        assert rc == -1 and "precond_variant" in msg
    for v in (-1, 5):
        rc, _, msg = _setup(lib, 2, 4, rp, ci, va, off, P.default_params(2, spmv_lane_shift=v))
        assert rc == -1 and "spmv_lane_shift" in msg
    rc, _, msg = _setup(lib, 2, 4, rp, ci, va, off, P.default_params(2, spmv_stage=2))
    assert rc == -1 and "spmv_stage" in msg
    assert P.default_params(2).spmv_order == 1
    rc, _, msg = _setup(lib, 2, 4, rp, ci, va, off, P.default_params(2, spmv_order=2))
    assert rc == -1 and "spmv_order" in msg


def test_null_context_calls(lib):
    assert lib.fsi_precond_build(None, 0, None) == -1
    assert lib.fsi_solve(None, None, None, 1e-8, None) == -1
    lib.fsi_free(None)


def test_learned_defaults_and_validation(lib):
    import paper_1801_05648_gb300 as P
    assert P.default_params(2).learned_accept == pytest.approx(0.1)
    tp = P.default_train_params()
    assert (tp.lr, tp.beta1, tp.beta2, tp.eps, tp.weight_decay, tp.init_out_scale) == \
        (1e-3, 0.9, 0.999, 1e-8, 0.0, 0.01)
    assert list(tp.sigma_in) == [1.0] * 5 and list(tp.sigma_out) == [1.0] * 5
    rp, ci, va, off = _tiny_csr()
    for bad in (0.0, 1.5, float("nan")):
        rc, _, msg = _setup(lib, 2, 4, rp, ci, va, off, P.default_params(2, learned_accept=bad))
        assert rc == -1 and "learned_accept" in msg
    # trainer parameters are checked before any device memory is touched
    h = ctypes.c_void_p()
    rc = lib.fsi_trainer_create(ctypes.byref(h), ctypes.byref(P.default_train_params(sigma_in=[1, 0, 1, 1, 1])))
    assert rc == -1 and not h.value and "scales" in lib.fsi_last_error(None).decode()
    rc = lib.fsi_trainer_create(ctypes.byref(h), ctypes.byref(P.default_train_params(beta1=1.0)))
    assert rc == -1 and "AdamW" in lib.fsi_last_error(None).decode()
    assert tp.dim == 2
    rc = lib.fsi_trainer_create(ctypes.byref(h), ctypes.byref(P.default_train_params(dim=4)))
    assert rc == -1 and not h.value and "dim" in lib.fsi_last_error(None).decode()


def test_mlp_sizes_agree_with_the_oracle_layout():
    """The header's parameter and input counts (2D and 3D) against the oracle's layout."""
    import paper_1801_05648_gb300 as P
    from oracle import learned as L
    hdr = open(os.path.join(ROOT, "include", "fsi.h")).read()
    defs = dict(re.findall(r"#define (FSI_MLP_\w+) (\d+)", hdr))
    assert int(defs["FSI_MLP_PARAMS"]) == P.FSI_MLP_PARAMS == L.N_PARAMS == P.mlp_params(2)
    assert int(defs["FSI_MLP_PARAMS_3D"]) == P.FSI_MLP_PARAMS_3D == L.N_PARAMS_3D == P.mlp_params(3)
    assert int(defs["FSI_MLP_INPUTS"]) == L.layout(2)[0] == P.mlp_inputs(2)
    assert int(defs["FSI_MLP_INPUTS_3D"]) == L.layout(3)[0] == P.mlp_inputs(3)


def test_learned_null_calls(lib):
    assert lib.fsi_learned_setup(None, 1, None, None) == -1
    assert lib.fsi_learned_load(None, b"x") == -1
    assert lib.fsi_learned_set_weights(None, None, None, None) == -1
    assert lib.fsi_learned_apply(None, None, None) == -1
    assert lib.fsi_learned_features(None, None, None, None) == -1
    assert lib.fsi_set_harvest(None, None, 0) == -1
    assert lib.fsi_set_flags(None, 0) == -1
    assert lib.fsi_set_learned_accept(None, 0.5) == -1
    assert lib.fsi_trainer_create(None, None) == -1
    assert lib.fsi_trainer_step(None, None, None, None) == -1
    assert lib.fsi_trainer_loss(None, None, None, None) == -1
    assert lib.fsi_trainer_update(None, None, 0.0) == -1
    assert lib.fsi_trainer_set_master(None, None) == -1
    assert lib.fsi_trainer_get(None, None, None, None) == -1
    assert lib.fsi_trainer_save(None, b"x") == -1
    lib.fsi_trainer_free(None)


def test_committed_weights_file_is_well_formed():
    from oracle import learned as L
    path = os.path.join(ROOT, "paper_1801_05648_gb300", "weights", "mlp_fsi2d_256x128.bin")
    bits, si, so = L.read_weights(path)
    assert bits.shape == (L.N_PARAMS,) and np.all(np.isfinite(L.bf16_value(bits)))
    assert np.all(si > 0) and np.all(so > 0)


def _header_struct_fields(name):
    text = open(os.path.join(ROOT, "include", "fsi.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct " + name + r"\s*\{(.*?)\}\s*" + name + ";", text, flags=re.S).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        # "int presmooth, postsmooth" / "const double* relres_hist" / "float sigma_in[5]"
        head, *rest = [d.strip() for d in decl.split(",")]
        fields.append(re.sub(r"\[.*\]", "", head.split()[-1]).lstrip("*"))
        fields += [re.sub(r"\[.*\]", "", r).lstrip("*") for r in rest]
    return fields


@pytest.mark.parametrize("cname,pyname", [("fsi_params", "Params"), ("fsi_stats", "Stats"),
                                          ("fsi_asm_mesh", "AsmMesh"), ("fsi_asm_physics", "AsmPhysics")])
def test_binding_structs_follow_the_header(cname, pyname):
    """The ctypes mirrors list the C structs' fields in the header's order (a
    field added to one side only would shift every later field)."""
    from paper_1801_05648_gb300 import fsi
    py = [f[0] for f in getattr(fsi, pyname)._fields_]
    assert py == _header_struct_fields(cname)


def test_binding_constants_follow_the_header():
    """Every FSI_* enumerator of include/fsi.h has the same value in the binding."""
    from paper_1801_05648_gb300 import fsi
    text = open(os.path.join(ROOT, "include", "fsi.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    consts = dict((k, int(v)) for k, v in re.findall(r"\b(FSI_[A-Z0-9_]+)\s*=\s*(-?\d+)", text))
    assert len(consts) >= 20
    for k, v in consts.items():
        assert getattr(fsi, k) == v, k
