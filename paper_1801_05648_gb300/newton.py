"""Quasi-Newton time step of the monolithic FSI system (Alg. 1 with the solver
settings of Sec. 6): each Newton correction solves J(U_k) dU = -R(U_k) with
FGMRES and the block preconditioner of Alg. 2 on the GPU; the Jacobian (and the
preconditioner built from it) is re-assembled only when the last iteration
reduced the residual by less than a factor 10, ||r_k||_inf > 0.1 ||r_{k-1}||_inf;
the iteration stops at ||r_k||_inf < 1e-6 ||r_0||_inf; each linear solve runs to
a relative residual of 1e-3 (a reduction by 10^3).

``newton_step`` assembles residual and Jacobian on the host with ``fsigen``
(forward-mode dual numbers) and runs the linear solves through
``fsi.FSISolver``; ``solver_factory`` replaces the GPU solver (e.g. by a sparse
direct solve on the CPU) when the quasi-Newton logic itself is what is being
exercised.  ``newton_step_device`` keeps the whole loop on the GPU: residual and
Jacobian from ``fsi.FSIAssembler`` (device assembly), the new Jacobian handed to
the solver context on the device (``fsi_update_values``), the update U += dU on
the device; only ||R||_inf crosses to the host.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import fsi


@dataclass
class NewtonResult:
    U: np.ndarray
    converged: bool
    iterations: int
    assemblies: int
    residuals: list = field(default_factory=list)     # ||r_k||_inf, k = 0, 1, ...
    linear_iters: list = field(default_factory=list)  # FGMRES iterations per correction
    seconds: float = 0.0                              # wall time of the iteration (device loop)


def gpu_solver_factory(precision: str = "fp32", **params):
    """Factory for the GPU linear solve: build(pb, vals) -> solve(rhs) -> dU.
    ``params`` go to ``fsi.default_params`` (dt_theta defaults to dt * theta of
    the problem's configuration)."""
    import torch

    def build(pb, vals):
        prm = dict(params)
        prm.setdefault("dt_theta", pb.cfg.dt * pb.cfg.theta)
        prm.setdefault("mass_ratio", 8.0 if pb.dim == 2 else 20.0)
        prm.setdefault("flags", fsi.FSI_USE_GRAPHS)
        S = fsi.FSISolver(pb.dim, pb.rowptr, pb.colind, vals, pb.offsets, pb.solid_node_coords(),
                          fsi.default_params(pb.dim, **prm))
        S.precond_build(precision)

        def solve(rhs, rtol):
            b = torch.tensor(rhs, device="cuda")
            x = torch.zeros_like(b)
            st = S.solve(b, x, rtol)
            return x.cpu().numpy(), st.iters

        solve.close = S.close
        return solve

    return build


def newton_step(pb, U0, Uold, solver_factory=None, rtol_linear=1e-3, tol=1e-6, reassemble_above=0.1,
                max_iter=30, fixed_values=None) -> NewtonResult:
    """Newton iteration for one time step from the initial guess U0 (previous
    step Uold).  ``fixed_values`` (indices, values) are Dirichlet data imposed on
    U before the first residual (e.g. an inflow profile); the Jacobian rows of
    fixed DOFs are identity rows, so corrections keep them."""
    factory = solver_factory or gpu_solver_factory()
    U = np.array(U0, dtype=np.float64)
    if fixed_values is not None:
        idx, val = fixed_values
        U[idx] = val
    R = pb.residual(U, Uold)
    r0 = float(np.max(np.abs(R)))
    res = NewtonResult(U, r0 == 0.0, 0, 0, [r0])
    solve = None
    prev = None
    try:
        while res.residuals[-1] >= tol * r0 and res.iterations < max_iter and r0 > 0.0:
            rk = res.residuals[-1]
            if solve is None or rk > reassemble_above * prev:
                if solve is not None and hasattr(solve, "close"):
                    solve.close()
                solve = factory(pb, pb.jacobian(U, Uold))
                res.assemblies += 1
            dU, iters = solve(-R, rtol_linear)
            res.linear_iters.append(int(iters))
            U = U + dU
            R = pb.residual(U, Uold)
            prev = rk
            res.iterations += 1
            res.residuals.append(float(np.max(np.abs(R))))
    finally:
        if solve is not None and hasattr(solve, "close"):
            solve.close()
    res.U = U
    res.converged = res.residuals[-1] < tol * r0 or r0 == 0.0
    return res


def newton_step_device(pb, U0, Uold, precision: str = "fp32", rtol_linear=1e-3, tol=1e-6, reassemble_above=0.1,
                       max_iter=30, fixed_values=None, **params) -> NewtonResult:
    """The quasi-Newton iteration of ``newton_step`` with assembly, solves and
    updates on the device.  Each correction solves J dU = R and applies U -= dU."""
    import time
    import torch
    stream = torch.cuda.Stream()
    U = np.array(U0, dtype=np.float64)
    if fixed_values is not None:
        idx, val = fixed_values
        U[idx] = val
    asm = fsi.FSIAssembler.from_problem(pb, stream=stream)
    prm = dict(params)
    prm.setdefault("dt_theta", pb.cfg.dt * pb.cfg.theta)
    prm.setdefault("mass_ratio", 8.0 if pb.dim == 2 else 20.0)
    prm.setdefault("flags", fsi.FSI_USE_GRAPHS)
    S = fsi.FSISolver(pb.dim, pb.rowptr, pb.colind, None, pb.offsets, pb.solid_node_coords(),
                      fsi.default_params(pb.dim, **prm), stream=stream)
    dev = torch.device("cuda")
    with torch.cuda.stream(stream):
        Ud = torch.tensor(U, device=dev)
        Uo = torch.tensor(np.asarray(Uold, np.float64), device=dev)
        R = torch.empty_like(Ud)
        dU = torch.zeros_like(Ud)
        vals = torch.empty(int(pb.rowptr[-1]), dtype=torch.float64, device=dev)
    stream.synchronize()
    t0 = time.perf_counter()
    try:
        _, r0 = asm.residual(Ud, Uo, R)
        res = NewtonResult(None, r0 == 0.0, 0, 0, [r0])
        prev = None
        while res.residuals[-1] >= tol * r0 and res.iterations < max_iter and r0 > 0.0:
            rk = res.residuals[-1]
            if res.assemblies == 0 or rk > reassemble_above * prev:
                asm.jacobian(Ud, Uo, vals)
                S.update_values(vals)
                S.precond_build(precision)
                res.assemblies += 1
            st = S.solve(R, dU, rtol_linear)
            res.linear_iters.append(int(st.iters))
            asm.axpy(-1.0, dU, Ud)
            _, r = asm.residual(Ud, Uo, R)
            prev = rk
            res.iterations += 1
            res.residuals.append(r)
        stream.synchronize()
        res.seconds = time.perf_counter() - t0
        res.U = Ud.cpu().numpy()
    finally:
        S.close()
        asm.close()
    res.converged = res.residuals[-1] < tol * r0 or r0 == 0.0
    return res
