"""Seeded input generator for the monolithic FSI linear solve.

Builds the linearised ALE fluid-structure Jacobian A_h (Eq. mat:small, Sec. 3.4)
of the semilinear form Eq. (fsi:all) at a seeded smooth state, plus a seeded
right-hand side, on structured box meshes that stand in for the paper's 2D
channel (Sec. 6.1) and 3D obstacle (Sec. 6.2) cases.  The C++ part
(``assemble.cpp``) does the finite-element work; this module compiles it, draws
the seeded state and right-hand side, and hands out plain numpy arrays.

Both the CPU oracle and the CUDA library take what this module returns as input.
It holds none of the solver's arithmetic (no Krylov, AMG or preconditioner step).

Input recipe (seeded, synthetic):
  * state: for each scalar field in the order v_0..v_{d-1}, u_0..u_{d-1}, p, with
    ``rng = numpy.random.default_rng(state_seed)`` shared across fields, draw
    ``modes = rng.integers(1, 5, size=(4, d))`` and ``a = rng.uniform(-1, 1, 4)``;
    the field is ``A * sum_k a_k prod_j sin(pi m_kj x_j / L_j) / sum_k |a_k|``
    evaluated at the DOF's node (zero on the whole outer boundary, |f| <= A);
  * previous time step: U^{n-1} = U ("rest", the default: the mesh velocity
    (u - u^{n-1})/dt vanishes) or U^{n-1} = 0 ("zero");
  * right-hand side ("manufactured", the default): b = A x* with
    ``x* = numpy.random.default_rng(rhs_seed).standard_normal(n)`` zeroed on
    fixed (identity) rows, so x* is the exact solution; ("normal"): b itself is
    that N(0,1) draw zeroed on fixed rows.  With the normal draw the unscaled
    equations (mass rows ~h^2, pressure rows ~h, solid stiffness rows ~1e4)
    force solution components near 1e10 and the FP64 rounding floor of
    ||b - A x|| / ||b|| reaches ~1e-8 from 128x64 cells on (a sparse direct
    solve gives 1.04e-8 there), so a 1e-8 tolerance is unattainable.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "assemble.cpp")
_SO = os.path.join(_HERE, "libfsigen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``assemble.cpp`` into ``libfsigen.so`` (g++, OpenMP, no FMA contraction
    so x86 and Arm hosts produce the same bits)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["g++", "-O3", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("L", ctypes.c_double * 3),
                ("solid_h", ctypes.c_double), ("rho_f", ctypes.c_double), ("nu_f", ctypes.c_double),
                ("mu_s", ctypes.c_double), ("lambda_s", ctypes.c_double), ("rho_s", ctypes.c_double),
                ("dt", ctypes.c_double), ("theta", ctypes.c_double), ("pressure", ctypes.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            vp, i64p, i32p, f64p, u8p = (ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_uint8))
            lib.fsigen_create.restype = vp
            lib.fsigen_create.argtypes = [ctypes.POINTER(_Params)]
            lib.fsigen_free.argtypes = [vp]
            lib.fsigen_sizes.argtypes = [vp, i64p]
            lib.fsigen_pattern.argtypes = [vp, i64p, i32p]
            lib.fsigen_dof_info.argtypes = [vp, f64p, i32p, i32p, u8p]
            lib.fsigen_jacobian.argtypes = [vp, f64p, f64p, f64p, f64p]
            lib.fsigen_jacobian.restype = ctypes.c_int
            lib.fsigen_residual.argtypes = [vp, f64p, f64p, f64p, f64p]
            lib.fsigen_residual.restype = ctypes.c_int
            lib.fsigen_num_threads.restype = ctypes.c_int
            lib.fsigen_node_map.argtypes = [vp, i32p, i32p]
            lib.fsigen_node_map.restype = ctypes.c_int
            lib.fsigen_cell_map.argtypes = [vp, i32p, ctypes.POINTER(ctypes.c_uint32)]
            lib.fsigen_cell_map.restype = None
            _lib = lib
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


@dataclass(frozen=True)
class FSIConfig:
    """Mesh, material and seed parameters of one synthetic Jacobian.

    Material values are the FSI-2 set of Sec. 6.1 (fluid density 1e3, viscosity
    1e-3, solid density 1e4, Lame mu 0.5e6, lambda 2e6); dt = 0.01 and the theta
    scheme of Sec. 3.2 with 0 < theta <= 1 (1: backward Euler, the default; 1/2:
    Crank-Nicolson; 1/2 + dt: shifted).  A solve of such a Jacobian uses
    dt_theta = dt * theta in its preconditioner.
    """
    name: str
    dim: int
    n: tuple
    L: tuple = (2.0, 1.0, 1.0)
    solid_h: float = 0.25
    amplitude: float = 1e-2
    state_seed: int = 0
    rhs_seed: int = 0
    rho_f: float = 1e3
    nu_f: float = 1e-3
    mu_s: float = 5e5
    lambda_s: float = 2e6
    rho_s: float = 1e4
    dt: float = 0.01
    theta: float = 1.0
    prev_state: str = "rest"      # U^{n-1} = U ("rest") or 0 ("zero")
    rhs_kind: str = "manufactured"  # b = A x*, x* ~ N(0,1) ("manufactured") or b ~ N(0,1) ("normal")
    pressure: str = "q1"          # "q1": continuous Q1 pressure; "p1disc": discontinuous P1 per fluid cell (Sec. 3.4)

    def with_(self, **kw) -> "FSIConfig":
        return replace(self, **kw)


CONFIGS = {
    # 16x16 cells on [0,2]x[0,1], solid strip y < 0.25: n = 4,645
    "2d_tiny": FSIConfig("2d_tiny", 2, (16, 16)),
    # 256x128 cells: n = 560,517
    "2d_mid": FSIConfig("2d_mid", 2, (256, 128)),
    # 512x256 cells: n = 2,235,141 (kernel profiles above L2 size, a few GB on the device)
    "2d_512x256": FSIConfig("2d_512x256", 2, (512, 256)),
    # 32x16x16 hex cells on [0,2]x[0,1]^2, solid slab z < 0.25: n = 434,247
    "3d": FSIConfig("3d", 3, (32, 16, 16)),
    # 1024x512 cells: n = 8,926,725.  Run at amplitude 1e-2: at 5e-2 the seed-0
    # state compresses the solid past the stability limit of the St. Venant-
    # Kirchhoff law (indefinite solid block, see the next entry)
    "2d_large": FSIConfig("2d_large", 2, (1024, 512)),
    "2d_large_amp5e-2": FSIConfig("2d_large_amp5e-2", 2, (1024, 512), amplitude=5e-2),
    # the paper's Q2-Q2-P1disc element (Sec. 3.4) on the 256x128 mesh: 3 pressure DOFs per fluid cell
    "2d_mid_p1disc": FSIConfig("2d_mid_p1disc", 2, (256, 128), pressure="p1disc"),
}


class Problem:
    """Mesh, DOF classes and sparsity pattern of one configuration."""

    def __init__(self, cfg: FSIConfig):
        lib = _load()
        self.cfg = cfg
        p = _Params()
        p.dim = cfg.dim
        for d in range(3):
            p.n[d] = cfg.n[d] if d < cfg.dim else 1
            p.L[d] = cfg.L[d]
        p.solid_h, p.rho_f, p.nu_f = cfg.solid_h, cfg.rho_f, cfg.nu_f
        p.mu_s, p.lambda_s, p.rho_s, p.dt, p.theta = cfg.mu_s, cfg.lambda_s, cfg.rho_s, cfg.dt, cfg.theta
        if cfg.pressure not in ("q1", "p1disc"):
            raise ValueError(f"unknown pressure space {cfg.pressure!r}")
        p.pressure = 1 if cfg.pressure == "p1disc" else 0
        self._h = lib.fsigen_create(ctypes.byref(p))
        if not self._h:
            raise ValueError(f"fsigen: invalid configuration {cfg}")
        sizes = np.zeros(9, np.int64)
        lib.fsigen_sizes(self._h, _ptr(sizes, ctypes.c_int64))
        self.offsets = sizes[:6].copy()
        self.n = int(sizes[5])
        self.nnz = int(sizes[6])
        self.n_q2, self.n_q1 = int(sizes[7]), int(sizes[8])
        self.dim = cfg.dim
        self.rowptr = np.empty(self.n + 1, np.int64)
        self.colind = np.empty(self.nnz, np.int32)
        lib.fsigen_pattern(self._h, _ptr(self.rowptr, ctypes.c_int64), _ptr(self.colind, ctypes.c_int32))
        self.coords = np.empty((self.n, self.dim), np.float64)
        self.field = np.empty(self.n, np.int32)
        self.comp = np.empty(self.n, np.int32)
        self.fixed = np.empty(self.n, np.uint8)
        lib.fsigen_dof_info(self._h, _ptr(self.coords, ctypes.c_double), _ptr(self.field, ctypes.c_int32),
                            _ptr(self.comp, ctypes.c_int32), _ptr(self.fixed, ctypes.c_uint8))
        self.fixed = self.fixed.astype(bool)

    def __del__(self):
        if getattr(self, "_h", None):
            _load().fsigen_free(self._h)
            self._h = None

    # ------------------------------------------------------------ seeded data
    def seeded_state(self, seed: int | None = None, amplitude: float | None = None) -> np.ndarray:
        """Smooth state U: per scalar field a normalised sum of 4 random sine modes."""
        cfg = self.cfg
        seed = cfg.state_seed if seed is None else seed
        A = cfg.amplitude if amplitude is None else amplitude
        d = self.dim
        rng = np.random.default_rng(seed)
        U = np.zeros(self.n)
        L = np.asarray(cfg.L[:d])
        for fld, ncomp in ((0, d), (1, d), (2, 1)):
            for c in range(ncomp):
                modes = rng.integers(1, 5, size=(4, d))
                a = rng.uniform(-1.0, 1.0, size=4)
                sel = (self.field == fld) & (self.comp == c)
                x = self.coords[sel]
                val = np.zeros(x.shape[0])
                for k in range(4):
                    term = np.full(x.shape[0], a[k])
                    for j in range(d):
                        term = term * np.sin(np.pi * modes[k, j] * x[:, j] / L[j])
                    val += term
                U[sel] = A * val / np.sum(np.abs(a))
        U[self.fixed] = 0.0
        return U

    def rhs(self, seed: int | None = None) -> np.ndarray:
        """The seeded N(0,1) draw, zeroed on fixed rows."""
        seed = self.cfg.rhs_seed if seed is None else seed
        b = np.random.default_rng(seed).standard_normal(self.n)
        b[self.fixed] = 0.0
        return b

    # --------------------------------------------------------------- assembly
    def jacobian(self, U: np.ndarray, Uold: np.ndarray | None = None) -> np.ndarray:
        """Values of dR/dU on the pattern (rowptr, colind)."""
        U = np.ascontiguousarray(U, np.float64)
        vals = np.empty(self.nnz, np.float64)
        minJ = ctypes.c_double(0.0)
        uo = None if Uold is None else np.ascontiguousarray(Uold, np.float64)
        rc = _load().fsigen_jacobian(self._h, _ptr(U, ctypes.c_double), _ptr(uo, ctypes.c_double),
                                     _ptr(vals, ctypes.c_double), ctypes.byref(minJ))
        self.min_J = minJ.value
        if rc == 1:
            raise RuntimeError("fsigen: Jacobian entry outside the sparsity pattern")
        if rc == 2:
            raise RuntimeError(f"fsigen: state folds the mesh (min J = {minJ.value})")
        return vals

    def residual(self, U: np.ndarray, Uold: np.ndarray | None = None) -> np.ndarray:
        U = np.ascontiguousarray(U, np.float64)
        R = np.empty(self.n, np.float64)
        minJ = ctypes.c_double(0.0)
        uo = None if Uold is None else np.ascontiguousarray(Uold, np.float64)
        rc = _load().fsigen_residual(self._h, _ptr(U, ctypes.c_double), _ptr(uo, ctypes.c_double),
                                     _ptr(R, ctypes.c_double), ctypes.byref(minJ))
        if rc == 2:
            raise RuntimeError(f"fsigen: state folds the mesh (min J = {minJ.value})")
        return R

    def node_map(self):
        """(node_dof [n_q2, 4] int32, patch [n_q2, 3^dim] int32).  node_dof rows: first
        v DOF, first u DOF, p DOF or -1, flags (1 solid closure, 2 v fixed, 4 u fixed,
        8 interface, 16 lattice i odd, 32 lattice j odd, 64 p row fixed, 128 lattice k
        odd); patch: the 3x3 (3x3x3) lattice neighbourhood of each Q2 node, direction 0
        fastest (-1 outside the mesh).  Nodal (Q1) pressure only."""
        nd = np.empty((self.n_q2, 4), np.int32)
        pt = np.empty((self.n_q2, 3 ** self.dim), np.int32)
        rc = _load().fsigen_node_map(self._h, _ptr(nd, ctypes.c_int32), _ptr(pt, ctypes.c_int32))
        if rc != 0:
            raise ValueError("node_map: nodal (Q1) pressure only")
        return nd, pt

    def cell_map(self):
        """(cell_dof [cells, NL] int32, cell_flags [cells] uint32): per cell (lexicographic,
        direction 0 fastest) the global DOF of each element DOF (v of Q2 node a comp i at
        a*dim + i, u at NQ2*dim + a*dim + i, pressure basis function P at 2*NQ2*dim + P:
        the Q1 vertices, or with P1disc the cell's d + 1 coefficients) and the
        flags bit 0 solid, bit 1 outflow-face fluid cell, bit 2 + a node a outside the
        closed solid region.  The mesh description a device assembler consumes."""
        n_cells = int(np.prod(self.cfg.n[:self.dim]))
        nq2 = 9 if self.dim == 2 else 27
        npres = self.dim + 1 if self.cfg.pressure == "p1disc" else 2 ** self.dim
        nl = 2 * nq2 * self.dim + npres
        cd = np.empty((n_cells, nl), np.int32)
        cf = np.empty(n_cells, np.uint32)
        _load().fsigen_cell_map(self._h, _ptr(cd, ctypes.c_int32), _ptr(cf, ctypes.c_uint32))
        return cd, cf

    def solid_node_coords(self) -> np.ndarray:
        """Coordinates of the s_v nodes (one row per node, s_v node order)."""
        lo, hi = self.offsets[1], self.offsets[2]
        return np.ascontiguousarray(self.coords[lo:hi:self.dim])


@dataclass
class System:
    """One linear system A x = b in monolithic CSR with its class offsets."""
    cfg: FSIConfig
    dim: int
    rowptr: np.ndarray
    colind: np.ndarray
    vals: np.ndarray
    offsets: np.ndarray
    rhs: np.ndarray
    solid_coords: np.ndarray
    fixed: np.ndarray
    state: np.ndarray = field(repr=False, default=None)
    x_exact: np.ndarray = field(repr=False, default=None)   # manufactured solution (None for "normal")

    @property
    def n(self) -> int:
        return int(self.offsets[5])

    def scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.vals, self.colind, self.rowptr), shape=(self.n, self.n))


_problem_cache: dict = {}


def get_problem(cfg: FSIConfig) -> Problem:
    key = (cfg.dim, tuple(cfg.n), tuple(cfg.L), cfg.solid_h, cfg.rho_f, cfg.nu_f, cfg.mu_s,
           cfg.lambda_s, cfg.rho_s, cfg.dt, cfg.theta, cfg.pressure)
    if key not in _problem_cache:
        _problem_cache[key] = Problem(cfg)
    return _problem_cache[key]


def make_system(cfg: FSIConfig | str, state_seed: int | None = None, rhs_seed: int | None = None) -> System:
    """Assemble the seeded Jacobian and right-hand side of a configuration."""
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    if state_seed is not None:
        cfg = cfg.with_(state_seed=state_seed)
    if rhs_seed is not None:
        cfg = cfg.with_(rhs_seed=rhs_seed)
    pb = get_problem(cfg)
    U = pb.seeded_state(cfg.state_seed, cfg.amplitude)
    if cfg.prev_state == "rest":
        Uold = U.copy()
    elif cfg.prev_state == "zero":
        Uold = None
    else:
        raise ValueError(f"unknown prev_state {cfg.prev_state!r}")
    vals = pb.jacobian(U, Uold)
    draw = pb.rhs(cfg.rhs_seed)
    x_exact = None
    if cfg.rhs_kind == "manufactured":
        import scipy.sparse as sp
        A = sp.csr_matrix((vals, pb.colind, pb.rowptr), shape=(pb.n, pb.n))
        x_exact = draw
        b = A @ x_exact
    elif cfg.rhs_kind == "normal":
        b = draw
    else:
        raise ValueError(f"unknown rhs_kind {cfg.rhs_kind!r}")
    return System(cfg=cfg, dim=pb.dim, rowptr=pb.rowptr, colind=pb.colind, vals=vals,
                  offsets=pb.offsets.copy(), rhs=b, solid_coords=pb.solid_node_coords(),
                  fixed=pb.fixed, state=U, x_exact=x_exact)
