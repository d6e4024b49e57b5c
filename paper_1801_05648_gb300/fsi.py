"""Thin ctypes binding of libfsi.so (declared in include/fsi.h).

Argument marshalling only: every step of the solve runs in the CUDA library.
PyTorch supplies device memory (float64 CUDA tensors) and the stream.  A missing
or unloadable library raises immediately; there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfsi.so")

FSI_OK, FSI_EINVAL, FSI_ENOMEM, FSI_ECUDA, FSI_ENOTCONV, FSI_EBREAKDOWN, FSI_ENONFINITE = 0, -1, -2, -3, -4, -5, -6
FSI_FP64, FSI_FP32_AMG = 0, 1
FSI_X0_GIVEN, FSI_USE_GRAPHS, FSI_NO_RIGID_MODES, FSI_CLUSTER_COARSE, FSI_LEARNED, FSI_NO_PDL = 1, 2, 4, 8, 16, 32
FSI_GRID_COARSE, FSI_FLUID_GMRES, FSI_MLP_CUDA_CORES = 64, 128, 256
FSI_PRECOND_LDU, FSI_PRECOND_LOWER, FSI_PRECOND_UPPER, FSI_PRECOND_DIAG = 0, 1, 2, 3
FSI_MLP_PARAMS, FSI_MLP_INPUTS = 7941, 53
FSI_MLP_PARAMS_3D, FSI_MLP_INPUTS_3D = 17543, 201


def mlp_params(dim: int) -> int:
    """Parameter count of the learned stage's MLP on a mesh of dimension dim."""
    return FSI_MLP_PARAMS_3D if dim == 3 else FSI_MLP_PARAMS


def mlp_inputs(dim: int) -> int:
    """Input width of the learned stage's MLP on a mesh of dimension dim."""
    return FSI_MLP_INPUTS_3D if dim == 3 else FSI_MLP_INPUTS
STATUS_NAMES = {0: "FSI_OK", -1: "FSI_EINVAL", -2: "FSI_ENOMEM", -3: "FSI_ECUDA", -4: "FSI_ENOTCONV",
                -5: "FSI_EBREAKDOWN", -6: "FSI_ENONFINITE"}
BLOCKS = {"mesh": 0, "solid_schur": 1, "fluid_velocity": 2, "pressure_schur": 3, "solid_mass": 4,
          "solid": 5, "fluid": 6, "precond": 7}

# Every symbol include/fsi.h declares.
EXPORTED = ["fsi_default_params", "fsi_setup", "fsi_precond_build", "fsi_solve", "fsi_free", "fsi_last_error",
            "fsi_apply_operator", "fsi_apply_block", "fsi_smoother_step", "fsi_amg_info", "fsi_amg_export",
            "fsi_mass_solve_noalloc", "fsi_learned_setup", "fsi_learned_load", "fsi_learned_set_weights",
            "fsi_learned_apply", "fsi_learned_features", "fsi_set_harvest", "fsi_default_train_params",
            "fsi_trainer_create", "fsi_trainer_step", "fsi_trainer_loss", "fsi_trainer_update",
            "fsi_trainer_set_master", "fsi_trainer_get", "fsi_trainer_save", "fsi_trainer_free", "fsi_set_flags",
            "fsi_set_learned_accept", "fsi_update_values", "fsi_asm_create", "fsi_asm_residual",
            "fsi_asm_jacobian", "fsi_asm_axpy", "fsi_asm_last_error", "fsi_asm_free", "fsi_check_device_errors",
            "fsi_debug_inject"]

# fault-injection bits of fsi_debug_inject (tests of the bounded waits)
FSI_INJECT_COARSE_BARRIER, FSI_INJECT_MLP_COMMIT = 1, 2


class FSIError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("maxit", ctypes.c_int), ("flags", ctypes.c_int),
                ("dt_theta", ctypes.c_double), ("strength_theta", ctypes.c_double), ("coarse_max", ctypes.c_int),
                ("max_levels", ctypes.c_int), ("cheb_degree", ctypes.c_int), ("cheb_ratio", ctypes.c_double),
                ("cheb_upper", ctypes.c_double), ("power_iters", ctypes.c_int), ("drop_tol", ctypes.c_double),
                ("presmooth", ctypes.c_int), ("postsmooth", ctypes.c_int), ("vcycles_mesh", ctypes.c_int),
                ("vcycles_solid", ctypes.c_int), ("vcycles_fluid", ctypes.c_int),
                ("vcycles_pressure", ctypes.c_int), ("mass_degree", ctypes.c_int), ("mass_ratio", ctypes.c_double),
                ("spmv_unroll", ctypes.c_int),
                ("learned_accept", ctypes.c_double), ("spmv_prefetch", ctypes.c_int),
                ("cluster_max_bytes", ctypes.c_double), ("cheb_degree_coarse", ctypes.c_int),
                ("fluid_gmres_iters", ctypes.c_int), ("precond_variant", ctypes.c_int),
                ("spmv_lane_shift", ctypes.c_int), ("spmv_stage", ctypes.c_int),
                ("spmv_order", ctypes.c_int)]


class AsmMesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("pressure", ctypes.c_int), ("cells", ctypes.c_int * 3),
                ("h", ctypes.c_double * 3), ("n", ctypes.c_int64),
                ("cell_dof", ctypes.POINTER(ctypes.c_int32)), ("cell_flags", ctypes.POINTER(ctypes.c_uint32)),
                ("rowptr", ctypes.POINTER(ctypes.c_int64)), ("colind", ctypes.POINTER(ctypes.c_int32)),
                ("row_fixed", ctypes.POINTER(ctypes.c_uint8))]


class AsmPhysics(ctypes.Structure):
    _fields_ = [("rho_f", ctypes.c_double), ("nu_f", ctypes.c_double), ("mu_s", ctypes.c_double),
                ("lambda_s", ctypes.c_double), ("rho_s", ctypes.c_double), ("dt", ctypes.c_double),
                ("theta", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("cycles", ctypes.c_int), ("status", ctypes.c_int),
                ("true_relres", ctypes.c_double), ("setup_s", ctypes.c_double),
                ("precond_build_s", ctypes.c_double), ("solve_s", ctypes.c_double),
                ("operator_bytes", ctypes.c_double), ("precond_bytes", ctypes.c_double),
                ("relres_hist", ctypes.POINTER(ctypes.c_double)), ("hist_len", ctypes.c_int),
                ("kernel_launches", ctypes.c_int64), ("learned_accepted", ctypes.c_int),
                ("reorth_passes", ctypes.c_int)]


class TrainParams(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("weight_decay", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("init_out_scale", ctypes.c_double), ("sigma_in", ctypes.c_float * 5),
                ("sigma_out", ctypes.c_float * 5), ("dim", ctypes.c_int)]


@dataclass
class SolveStats:
    iters: int
    cycles: int
    status: int
    true_relres: float
    setup_s: float
    precond_build_s: float
    solve_s: float
    operator_bytes: float
    precond_bytes: float
    history: list
    kernel_launches: int
    learned_accepted: int = 0
    reorth_passes: int = 0


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libfsi.so (build it first with paper_1801_05648_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} is missing: run paper_1801_05648_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i64p, i32p, f64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32), \
        ctypes.POINTER(ctypes.c_double)
    lib.fsi_default_params.argtypes = [ctypes.POINTER(Params), ctypes.c_int]
    lib.fsi_default_params.restype = None
    lib.fsi_setup.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int64, i64p, i32p, f64p, i64p, f64p,
                              ctypes.POINTER(Params), vp]
    lib.fsi_setup.restype = ctypes.c_int
    lib.fsi_precond_build.argtypes = [vp, ctypes.c_int, ctypes.c_char_p]
    lib.fsi_precond_build.restype = ctypes.c_int
    lib.fsi_solve.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.POINTER(Stats)]
    lib.fsi_solve.restype = ctypes.c_int
    lib.fsi_free.argtypes = [vp]
    lib.fsi_free.restype = None
    lib.fsi_last_error.argtypes = [vp]
    lib.fsi_last_error.restype = ctypes.c_char_p
    lib.fsi_apply_operator.argtypes = [vp, vp, vp]
    lib.fsi_apply_operator.restype = ctypes.c_int
    lib.fsi_apply_block.argtypes = [vp, ctypes.c_int, vp, vp]
    lib.fsi_apply_block.restype = ctypes.c_int
    lib.fsi_smoother_step.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, f64p]
    lib.fsi_smoother_step.restype = ctypes.c_int
    lib.fsi_amg_info.argtypes = [vp, ctypes.c_int, ctypes.c_int, i64p, f64p]
    lib.fsi_amg_info.restype = ctypes.c_int
    lib.fsi_amg_export.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]
    lib.fsi_amg_export.restype = ctypes.c_int
    lib.fsi_mass_solve_noalloc.argtypes = [vp, vp, vp]
    lib.fsi_mass_solve_noalloc.restype = ctypes.c_int
    f32p, u16p = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_uint16)
    lib.fsi_learned_setup.argtypes = [vp, ctypes.c_int64, i32p, i32p]
    lib.fsi_learned_load.argtypes = [vp, ctypes.c_char_p]
    lib.fsi_learned_set_weights.argtypes = [vp, f32p, f32p, u16p]
    lib.fsi_learned_apply.argtypes = [vp, vp, vp]
    lib.fsi_learned_features.argtypes = [vp, vp, vp, vp]
    lib.fsi_set_harvest.argtypes = [vp, vp, ctypes.c_int]
    lib.fsi_default_train_params.argtypes = [ctypes.POINTER(TrainParams)]
    lib.fsi_default_train_params.restype = None
    lib.fsi_trainer_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(TrainParams)]
    lib.fsi_trainer_step.argtypes = [vp, vp, vp, f64p]
    lib.fsi_trainer_loss.argtypes = [vp, vp, vp, f64p]
    lib.fsi_trainer_update.argtypes = [vp, vp, ctypes.c_double]
    lib.fsi_set_flags.argtypes = [vp, ctypes.c_int]
    lib.fsi_check_device_errors.argtypes = [vp]
    lib.fsi_check_device_errors.restype = ctypes.c_int
    lib.fsi_debug_inject.argtypes = [vp, ctypes.c_int]
    lib.fsi_debug_inject.restype = ctypes.c_int
    lib.fsi_set_learned_accept.argtypes = [vp, ctypes.c_double]
    lib.fsi_trainer_set_master.argtypes = [vp, f32p]
    lib.fsi_trainer_get.argtypes = [vp, f32p, u16p, f32p]
    lib.fsi_trainer_save.argtypes = [vp, ctypes.c_char_p]
    lib.fsi_trainer_free.argtypes = [vp]
    lib.fsi_trainer_free.restype = None
    lib.fsi_update_values.argtypes = [vp, vp]
    lib.fsi_asm_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(AsmMesh), ctypes.POINTER(AsmPhysics), vp]
    lib.fsi_asm_residual.argtypes = [vp, vp, vp, vp, f64p, f64p]
    lib.fsi_asm_jacobian.argtypes = [vp, vp, vp, vp, f64p]
    lib.fsi_asm_axpy.argtypes = [vp, ctypes.c_double, vp, vp]
    lib.fsi_asm_last_error.argtypes = [vp]
    lib.fsi_asm_last_error.restype = ctypes.c_char_p
    lib.fsi_asm_free.argtypes = [vp]
    lib.fsi_asm_free.restype = None
    for name in ("fsi_update_values", "fsi_asm_create", "fsi_asm_residual", "fsi_asm_jacobian", "fsi_asm_axpy"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("fsi_learned_setup", "fsi_learned_load", "fsi_learned_set_weights", "fsi_learned_apply",
                 "fsi_learned_features", "fsi_set_harvest", "fsi_trainer_create", "fsi_trainer_step",
                 "fsi_trainer_loss", "fsi_trainer_update", "fsi_trainer_set_master", "fsi_trainer_get",
                 "fsi_trainer_save", "fsi_set_flags", "fsi_set_learned_accept"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


PEAKS_LIB_PATH = os.path.join(_HERE, "libfsi_peaks.so")
PEAKS_EXPORTED = ["fsi_probe_fma_rate"]


def probe_fma_rate(bits: int, iters: int = 4096, reps: int = 5):
    """Measured FMA throughput of the current device (libfsi_peaks.so, include/fsi_peaks.h):
    (FMAs per second, best launch ms) for bits = 64 or 32."""
    lib = ctypes.CDLL(PEAKS_LIB_PATH)
    lib.fsi_probe_fma_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]
    lib.fsi_probe_fma_rate.restype = ctypes.c_int
    rate, ms = ctypes.c_double(), ctypes.c_double()
    rc = lib.fsi_probe_fma_rate(int(bits), int(iters), int(reps), ctypes.byref(rate), ctypes.byref(ms))
    if rc != 0:
        raise FSIError(rc, "fsi_probe_fma_rate failed")
    return rate.value, ms.value


def default_params(dim: int, **overrides) -> Params:
    p = Params()
    load_library().fsi_default_params(ctypes.byref(p), dim)
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(f"unknown fsi_params field {k!r}")
        setattr(p, k, v)
    return p


def _np_ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _dev_ptr(t, n=None, dtype=None):
    """Device address of a contiguous CUDA tensor holding at least n entries
    (the library reads or writes n of them; a shorter tensor would be overrun)."""
    import torch
    dtype = torch.float64 if dtype is None else dtype
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"expected a contiguous {dtype} CUDA tensor")
    if n is not None and t.numel() < n:
        raise ValueError(f"tensor has {t.numel()} entries, the call needs {n}")
    return ctypes.c_void_p(t.data_ptr())


class FSISolver:
    """One monolithic Jacobian on the device: fsi_setup / fsi_precond_build / fsi_solve / fsi_free."""

    def __init__(self, dim, rowptr, colind, vals, offsets, node_coords=None, params: Params | None = None,
                 stream=None):
        lib = load_library()
        self._lib = lib
        self._h = ctypes.c_void_p()
        rowptr = np.ascontiguousarray(rowptr, np.int64)
        colind = np.ascontiguousarray(colind, np.int32)
        vals = None if vals is None else np.ascontiguousarray(vals, np.float64)   # None: pattern only
        offsets = np.ascontiguousarray(offsets, np.int64)
        self.n = int(offsets[5])
        self.nnz = int(rowptr[-1])
        self.dim = dim
        self.flags = int(params.flags) if params is not None else 0
        self.offsets = offsets.copy()
        coords = None if node_coords is None else np.ascontiguousarray(node_coords, np.float64)
        import torch
        # The library runs on its own (non-default) stream so that graph capture is
        # possible; every call first orders it after torch's current stream.
        self.stream = stream if stream is not None else torch.cuda.Stream()
        stream = self.stream.cuda_stream
        self._stream = stream
        self._order()
        rc = lib.fsi_setup(ctypes.byref(self._h), dim, self.n, _np_ptr(rowptr, ctypes.c_int64),
                           _np_ptr(colind, ctypes.c_int32), None if vals is None else _np_ptr(vals, ctypes.c_double),
                           _np_ptr(offsets, ctypes.c_int64),
                           None if coords is None else _np_ptr(coords, ctypes.c_double),
                           None if params is None else ctypes.byref(params), ctypes.c_void_p(stream))
        if rc != FSI_OK:
            raise FSIError(rc, lib.fsi_last_error(None).decode())

    @classmethod
    def from_system(cls, system, params=None, stream=None):
        return cls(system.dim, system.rowptr, system.colind, system.vals, system.offsets, system.solid_coords,
                   params, stream)

    def _check(self, rc):
        if rc != FSI_OK:
            raise FSIError(rc, self._lib.fsi_last_error(self._h).decode())

    def _order(self):
        import torch
        self.stream.wait_stream(torch.cuda.current_stream())

    def precond_build(self, precision: str | int = "fp64", learned_weights: str | None = None):
        prec = {"fp64": FSI_FP64, "fp32": FSI_FP32_AMG}.get(precision, precision)
        path = None if learned_weights is None else os.fsencode(learned_weights)
        self._check(self._lib.fsi_precond_build(self._h, int(prec), path))

    def solve(self, rhs, x, rtol=1e-8, raise_on_error=True) -> SolveStats:
        self._order()
        st = Stats()
        rc = self._lib.fsi_solve(self._h, _dev_ptr(rhs, self.n), _dev_ptr(x, self.n), rtol, ctypes.byref(st))
        hist = [st.relres_hist[i] for i in range(st.hist_len)] if st.hist_len else []
        out = SolveStats(st.iters, st.cycles, st.status, st.true_relres, st.setup_s, st.precond_build_s,
                         st.solve_s, st.operator_bytes, st.precond_bytes, hist, st.kernel_launches,
                         st.learned_accepted, st.reorth_passes)
        if rc != FSI_OK and raise_on_error:
            raise FSIError(rc, self._lib.fsi_last_error(self._h).decode())
        return out

    def apply_operator(self, x, y, sync=True):
        """y = A x (enqueued on the solver's stream; waits for it unless sync=False)."""
        self._order()
        self._check(self._lib.fsi_apply_operator(self._h, _dev_ptr(x, self.n), _dev_ptr(y, self.n)))
        if sync:
            self._sync()

    def apply_block(self, which, inp, out, sync=True):
        w = BLOCKS.get(which, which)
        n = self.block_size(w)
        self._order()
        self._check(self._lib.fsi_apply_block(self._h, int(w), _dev_ptr(inp, n), _dev_ptr(out, n)))
        if sync:
            self._sync()

    def _sync(self):
        self.stream.synchronize()

    def block_size(self, which) -> int:
        """Entries of the vectors fsi_apply_block(which) reads and writes (see BLOCKS)."""
        o = [int(v) for v in self.offsets]
        sizes = {0: o[1] - o[0], 1: o[2] - o[1], 2: o[4] - o[3], 3: o[5] - o[4], 4: o[3] - o[2],
                 5: o[3] - o[1], 6: o[5] - o[3], 7: self.n}
        w = BLOCKS.get(which, which)
        if w not in sizes:
            raise ValueError(f"unknown block {which!r}")
        return sizes[w]

    def mass_solve_noalloc(self, inp, out, sync=True):
        """A_uu^-1 in through fsi_mass_solve_noalloc (static device scratch, no allocation)."""
        self._order()
        n = self.block_size("solid_mass")
        self._check(self._lib.fsi_mass_solve_noalloc(self._h, _dev_ptr(inp, n), _dev_ptr(out, n)))
        if sync:
            self._sync()

    def smoother_steps(self, which, level, reps):
        """Enqueue `reps` Chebyshev SpMV steps on a hierarchy level (no wait); returns bytes per step."""
        b = ctypes.c_double()
        self._order()
        self._check(self._lib.fsi_smoother_step(self._h, BLOCKS.get(which, which), level, reps, ctypes.byref(b)))
        return b.value

    def amg_info(self, which, level=0):
        info = np.zeros(6, np.int64)
        lam = ctypes.c_double()
        self._check(self._lib.fsi_amg_info(self._h, BLOCKS.get(which, which), level, _np_ptr(info, ctypes.c_int64),
                                           ctypes.byref(lam)))
        return {"levels": int(info[0]), "nbrows": int(info[1]), "b": int(info[2]), "nnzb": int(info[3]),
                "nagg": int(info[4]), "ncoarse": int(info[5]), "lam": lam.value}

    def amg_export(self, which, level, what):
        """what: 'agg', 'A' (-> rowptr, colind, values) or 'P'."""
        w = BLOCKS.get(which, which)
        inf = self.amg_info(w, level)
        b = inf["b"]
        if what == "agg":
            out = np.empty(inf["nbrows"], np.int32)
            self._check(self._lib.fsi_amg_export(self._h, w, level, 0, out.ctypes.data_as(ctypes.c_void_p)))
            return out
        if what == "A":
            rp = np.empty(inf["nbrows"] + 1, np.int32)
            ci = np.empty(inf["nnzb"], np.int32)
            va = np.empty(inf["nnzb"] * b * b, np.float64)
            for k, arr in ((1, rp), (2, ci), (3, va)):
                self._check(self._lib.fsi_amg_export(self._h, w, level, k, arr.ctypes.data_as(ctypes.c_void_p)))
            return rp, ci, va.reshape(-1, b, b)
        if what == "P":
            nn = np.zeros(1, np.int64)
            self._check(self._lib.fsi_amg_export(self._h, w, level, 7, nn.ctypes.data_as(ctypes.c_void_p)))
            rp = np.empty(inf["nbrows"] + 1, np.int32)
            ci = np.empty(int(nn[0]), np.int32)
            self._check(self._lib.fsi_amg_export(self._h, w, level, 4, rp.ctypes.data_as(ctypes.c_void_p)))
            self._check(self._lib.fsi_amg_export(self._h, w, level, 5, ci.ctypes.data_as(ctypes.c_void_p)))
            va = np.empty(int(nn[0]) * b * 64, np.float64)   # k <= 6 (upper bound), trimmed below
            self._check(self._lib.fsi_amg_export(self._h, w, level, 6, va.ctypes.data_as(ctypes.c_void_p)))
            return rp, ci, va
        raise ValueError(what)

    def set_flags(self, flags: int):
        """Run-time flags (FSI_X0_GIVEN, FSI_USE_GRAPHS, FSI_LEARNED)."""
        self._check(self._lib.fsi_set_flags(self._h, int(flags)))
        self.flags = int(flags)

    def set_learned_accept(self, tau: float):
        """Accept the learned correction only when ||r' - A c|| < tau ||r'||."""
        self._check(self._lib.fsi_set_learned_accept(self._h, float(tau)))

    # ------------------------------------------------------------ learned stage
    def learned_setup(self, node_dof, patch):
        """Node map (host int32 arrays [n_nodes, 4] and [n_nodes, 3^dim]) for the learned stage."""
        nd = np.ascontiguousarray(node_dof, np.int32)
        pt = np.ascontiguousarray(patch, np.int32)
        slots = 3 ** self.dim
        if nd.ndim != 2 or nd.shape[1] != 4 or pt.shape != (nd.shape[0], slots):
            raise ValueError(f"node_dof must be [n_nodes, 4] and patch [n_nodes, {slots}]")
        self._check(self._lib.fsi_learned_setup(self._h, nd.shape[0], _np_ptr(nd, ctypes.c_int32),
                                                _np_ptr(pt, ctypes.c_int32)))
        self.n_nodes = int(nd.shape[0])

    def learned_load(self, path):
        self._check(self._lib.fsi_learned_load(self._h, os.fsencode(path)))

    def learned_set_weights(self, sigma_in, sigma_out, params_bf16):
        si = np.ascontiguousarray(sigma_in, np.float32)
        so = np.ascontiguousarray(sigma_out, np.float32)
        pb = np.ascontiguousarray(params_bf16, np.uint16)
        if si.shape != (5,) or so.shape != (5,) or pb.shape != (mlp_params(self.dim),):
            raise ValueError(f"sigma_in/sigma_out need 5 values and params {mlp_params(self.dim)} bfloat16 words")
        self._check(self._lib.fsi_learned_set_weights(self._h, _np_ptr(si, ctypes.c_float),
                                                      _np_ptr(so, ctypes.c_float), _np_ptr(pb, ctypes.c_uint16)))

    def learned_apply(self, r, c, sync=True):
        """c = MLP(r') (float64 device vectors of length n)."""
        if r.numel() != self.n or c.numel() != self.n:
            raise ValueError("r and c must have n entries")
        self._order()
        self._check(self._lib.fsi_learned_apply(self._h, _dev_ptr(r, self.n), _dev_ptr(c, self.n)))
        if sync:
            self._sync()

    def learned_features(self, r, feat, rho, sync=True):
        """Features [n_nodes, 53 (2D) or 201 (3D)] and rho [n_nodes] (float32 device tensors) of r'."""
        import torch
        nn = getattr(self, "n_nodes", None)
        if nn is None:
            raise RuntimeError("learned_setup first")
        ni = mlp_inputs(self.dim)
        if r.numel() != self.n or feat.numel() < nn * ni or rho.numel() < nn:
            raise ValueError(f"r needs n entries, feat n_nodes x {ni} and rho n_nodes")
        self._order()
        self._check(self._lib.fsi_learned_features(self._h, _dev_ptr(r, self.n),
                                                   _dev_ptr(feat, nn * ni, torch.float32),
                                                   _dev_ptr(rho, nn, torch.float32)))
        if sync:
            self._sync()

    def check_device_errors(self):
        """Wait for the context's stream; raise FSIError (FSI_ECUDA) if a bounded wait in a
        kernel gave up since the last check or solve."""
        self._check(self._lib.fsi_check_device_errors(self._h))

    def debug_inject(self, mask: int):
        """Fault injection for tests of the bounded waits (FSI_INJECT_*; 0 = none)."""
        self._check(self._lib.fsi_debug_inject(self._h, int(mask)))

    def set_harvest(self, buf=None, nvec=0):
        """Store r'_j = v_j - A P^-1 v_j of the first nvec iterations of later solves into buf [nvec, n]."""
        ptr = None if buf is None else _dev_ptr(buf, int(nvec) * self.n)
        if buf is not None and (buf.dim() != 2 or buf.shape[0] < nvec or buf.shape[1] != self.n):
            raise ValueError("buf must be [>= nvec, n]")
        self._keep_harvest = buf
        self._check(self._lib.fsi_set_harvest(self._h, ptr, int(nvec if buf is not None else 0)))

    def update_values(self, vals):
        """New operator values on the same CSR pattern (float64 CUDA tensor, nnz entries);
        precond_build must follow before the next solve."""
        nnz = getattr(self, "nnz", None)
        self._order()
        self._check(self._lib.fsi_update_values(self._h, _dev_ptr(vals, nnz)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.fsi_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class FSIAssembler:
    """fsi_asm: residual R(U) and Jacobian dR/dU of the ALE-FSI system on the device
    (include/fsi.h), for the Newton loop without host assembly.

    mesh: the cell map of a structured box mesh (cells per direction, cell size,
    element-DOF map, cell flags, the Jacobian's CSR pattern and fixed rows);
    physics: rho_f, nu_f, mu_s, lambda_s, rho_s, dt, theta."""

    def __init__(self, dim, cells, h, n, cell_dof, cell_flags, rowptr, colind, row_fixed, physics, stream=None,
                 pressure="q1"):
        import torch
        lib = load_library()
        self._lib = lib
        self._h = ctypes.c_void_p()
        self.n = int(n)
        self.dim = int(dim)
        self._keep = [np.ascontiguousarray(cell_dof, np.int32), np.ascontiguousarray(cell_flags, np.uint32),
                      np.ascontiguousarray(rowptr, np.int64), np.ascontiguousarray(colind, np.int32),
                      np.ascontiguousarray(row_fixed, np.uint8)]
        self.nnz = int(self._keep[2][-1])
        if pressure not in ("q1", "p1disc"):
            raise ValueError(f"unknown pressure space {pressure!r}")
        nq2 = 9 if self.dim == 2 else 27
        nl = 2 * nq2 * self.dim + (self.dim + 1 if pressure == "p1disc" else 2 ** self.dim)
        if self._keep[0].ndim != 2 or self._keep[0].shape[1] != nl:
            raise ValueError(f"cell_dof must be [cells, {nl}]")
        m = AsmMesh()
        m.dim = self.dim
        m.pressure = 1 if pressure == "p1disc" else 0
        for d in range(3):
            m.cells[d] = int(cells[d]) if d < dim else 1
            m.h[d] = float(h[d]) if d < dim else 1.0
        m.n = self.n
        m.cell_dof = _np_ptr(self._keep[0], ctypes.c_int32)
        m.cell_flags = _np_ptr(self._keep[1], ctypes.c_uint32)
        m.rowptr = _np_ptr(self._keep[2], ctypes.c_int64)
        m.colind = _np_ptr(self._keep[3], ctypes.c_int32)
        m.row_fixed = _np_ptr(self._keep[4], ctypes.c_uint8)
        ph = AsmPhysics(**{k: float(physics[k]) for k in ("rho_f", "nu_f", "mu_s", "lambda_s", "rho_s", "dt",
                                                           "theta")})
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.stream.wait_stream(torch.cuda.current_stream())
        rc = lib.fsi_asm_create(ctypes.byref(self._h), ctypes.byref(m), ctypes.byref(ph),
                                ctypes.c_void_p(self.stream.cuda_stream))
        self._keep = None                       # copied to the device
        if rc != FSI_OK:
            raise FSIError(rc, lib.fsi_asm_last_error(None).decode())

    @classmethod
    def from_problem(cls, pb, stream=None):
        """From a problem of the seeded input generator (its cell map, pattern and material)."""
        cfg = pb.cfg
        cd, cf = pb.cell_map()
        h = [cfg.L[d] / cfg.n[d] for d in range(pb.dim)]
        phys = dict(rho_f=cfg.rho_f, nu_f=cfg.nu_f, mu_s=cfg.mu_s, lambda_s=cfg.lambda_s, rho_s=cfg.rho_s,
                    dt=cfg.dt, theta=cfg.theta)
        return cls(pb.dim, cfg.n, h, pb.n, cd, cf, pb.rowptr, pb.colind, pb.fixed, phys, stream,
                   pressure=getattr(cfg, "pressure", "q1"))

    def _check(self, rc):
        if rc != FSI_OK:
            raise FSIError(rc, self._lib.fsi_asm_last_error(self._h).decode())

    def _order(self):
        import torch
        self.stream.wait_stream(torch.cuda.current_stream())

    def residual(self, U, Uold, R):
        """R = R(U) (float64 CUDA tensors of n entries; Uold None = 0); returns (min det F, max |R_i|)."""
        mj, rm = ctypes.c_double(), ctypes.c_double()
        self._order()
        self._check(self._lib.fsi_asm_residual(self._h, _dev_ptr(U, self.n),
                                               None if Uold is None else _dev_ptr(Uold, self.n), _dev_ptr(R, self.n),
                                               ctypes.byref(mj), ctypes.byref(rm)))
        return mj.value, rm.value

    def jacobian(self, U, Uold, vals):
        """vals = dR/dU in CSR order (float64 CUDA tensor of nnz entries); returns min det F."""
        mj = ctypes.c_double()
        self._order()
        self._check(self._lib.fsi_asm_jacobian(self._h, _dev_ptr(U, self.n),
                                               None if Uold is None else _dev_ptr(Uold, self.n),
                                               _dev_ptr(vals, self.nnz), ctypes.byref(mj)))
        return mj.value

    def axpy(self, alpha, x, y):
        """y += alpha x (float64 CUDA tensors of n entries)."""
        self._order()
        self._check(self._lib.fsi_asm_axpy(self._h, float(alpha), _dev_ptr(x, self.n), _dev_ptr(y, self.n)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.fsi_asm_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def default_train_params(**overrides) -> TrainParams:
    p = TrainParams()
    load_library().fsi_default_train_params(ctypes.byref(p))
    for k, v in overrides.items():
        if k in ("sigma_in", "sigma_out"):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = float(x)
        elif hasattr(p, k):
            setattr(p, k, v)
        else:
            raise KeyError(f"unknown fsi_train_params field {k!r}")
    return p


class Trainer:
    """fsi_trainer: AdamW training of the learned stage on residuals of FSISolver contexts."""

    def __init__(self, params: TrainParams | None = None, **overrides):
        lib = load_library()
        self._lib = lib
        self._h = ctypes.c_void_p()
        p = params if params is not None else default_train_params(**overrides)
        rc = lib.fsi_trainer_create(ctypes.byref(self._h), ctypes.byref(p))
        if rc != FSI_OK:
            raise FSIError(rc, lib.fsi_last_error(None).decode())
        self.n_params = mlp_params(p.dim)

    def _check_global(self, rc):
        if rc != FSI_OK:
            raise FSIError(rc, self._lib.fsi_last_error(None).decode())

    def step(self, solver: FSISolver, rprime) -> float:
        """Accumulate the gradient of ||r' - A c||^2 / ||r'||^2 for r' of `solver`; returns the loss."""
        if rprime.numel() != solver.n:
            raise ValueError("r' must have n entries")
        loss = ctypes.c_double()
        solver._order()
        rc = self._lib.fsi_trainer_step(self._h, solver._h, _dev_ptr(rprime, solver.n), ctypes.byref(loss))
        solver._check(rc)
        return loss.value

    def loss(self, solver: FSISolver, rprime) -> float:
        """Loss of r' with the current weights (no gradient)."""
        if rprime.numel() != solver.n:
            raise ValueError("r' must have n entries")
        loss = ctypes.c_double()
        solver._order()
        solver._check(self._lib.fsi_trainer_loss(self._h, solver._h, _dev_ptr(rprime, solver.n),
                                                 ctypes.byref(loss)))
        return loss.value

    def update(self, solver: FSISolver, lr: float = 0.0):
        """AdamW step with the mean accumulated gradient (lr <= 0: the creation-time rate)."""
        solver._check(self._lib.fsi_trainer_update(self._h, solver._h, float(lr)))

    def set_master(self, params):
        w = np.ascontiguousarray(params, np.float32)
        if w.shape != (self.n_params,):
            raise ValueError(f"params must hold {self.n_params} floats")
        self._check_global(self._lib.fsi_trainer_set_master(self._h, _np_ptr(w, ctypes.c_float)))

    def get(self):
        """(master float32, bfloat16 words, accumulated gradient float32)."""
        m = np.empty(self.n_params, np.float32)
        b = np.empty(self.n_params, np.uint16)
        g = np.empty(self.n_params, np.float32)
        self._check_global(self._lib.fsi_trainer_get(self._h, _np_ptr(m, ctypes.c_float),
                                                     _np_ptr(b, ctypes.c_uint16), _np_ptr(g, ctypes.c_float)))
        return m, b, g

    def save(self, path):
        self._check_global(self._lib.fsi_trainer_save(self._h, os.fsencode(path)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.fsi_trainer_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
