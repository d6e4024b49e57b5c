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


def test_default_params(lib):
    import paper_1801_05648_gb300 as P
    p2, p3 = P.default_params(2), P.default_params(3)
    assert (p2.restart, p2.maxit, p2.cheb_degree, p2.vcycles_solid, p2.mass_degree) == (100, 1000, 4, 2, 12)
    assert p2.mass_ratio == 8.0 and p3.mass_ratio == 20.0
    assert p2.strength_theta == 0.08 and p2.dt_theta == 0.01


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


def test_null_context_calls(lib):
    assert lib.fsi_precond_build(None, 0, None) == -1
    assert lib.fsi_solve(None, None, None, 1e-8, None) == -1
    lib.fsi_free(None)
