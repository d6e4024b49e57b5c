"""Training and evaluation driver of the learned correction stage.

The stage is trained on residual/error pairs that the method's own Newton-step
solves produce.  Trajectory: the generator's 2D channel (solid strip y < 0.25,
fluid above) started from rest and driven by a parabolic inflow on the fluid part
of x = 0, 6 y'(H - y') / H^2 s(t) vbar with y' = y - 0.25, fluid height H = 0.75,
vbar = 1 and the ramp s(t) = (1 - cos(pi t / 2)) / 2 of the FSI-2 benchmark
(Sec. 6.1); backward Euler (dt = 0.01), a few Newton steps per time step, each
Newton system J dU = -R (generator assembly on the host) solved by fsi_solve in
the FP32-AMG form.  Selected solves store their preconditioned residuals
r'_j = v_j - A P^-1 v_j (fsi_set_harvest); the stage is then trained on them by
the library's trainer (loss ||r' - A c(r')||^2 / ||r'||^2, the error of the
correction in the residual norm, on the system's own A).  This module only
orchestrates: assembly is the generator's, every solve, harvest, forward,
backward and AdamW step runs in libfsi's CUDA kernels.

    python -m paper_1801_05648_gb300.learned train --out weights.bin
    python -m paper_1801_05648_gb300.learned evaluate --weights weights.bin --config 2d_large
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time

import numpy as np

import fsigen

from . import fsi

DEFAULT_WEIGHTS = __file__.rsplit("/", 1)[0] + "/weights/mlp_fsi2d_256x128.bin"


def inflow(pb):
    """(DOF indices, profile values) of the inflow x-velocity on x = 0 above the solid."""
    h_s = pb.cfg.solid_h
    top = pb.cfg.L[1]
    x, y = pb.coords[:, 0], pb.coords[:, 1]
    sel = (pb.field == 0) & (pb.comp == 0) & (x == 0.0) & (y > h_s) & (y < top)
    H = top - h_s
    yp = y[sel] - h_s
    return np.nonzero(sel)[0], 6.0 * yp * (H - yp) / H ** 2


def ramp(t: float) -> float:
    return 0.5 * (1.0 - math.cos(math.pi * t / 2.0)) if t < 2.0 else 1.0


def newton_trajectory(cfg, steps, newton, solve, vbar=1.0):
    """Yield (step, k, vals, rhs, dU) for each Newton system along the trajectory;
    solve(vals, rhs) -> dU is the caller's GPU solve.  The state is advanced by dU."""
    pb = fsigen.get_problem(cfg)
    idx, prof = inflow(pb)
    U = np.zeros(pb.n)
    t = 0.0
    for step in range(steps):
        Uold = U.copy()
        t += cfg.dt
        U[idx] = prof * ramp(t) * vbar
        for k in range(newton):
            vals = pb.jacobian(U, Uold)
            rhs = -pb.residual(U, Uold)
            dU = solve(step, k, vals, rhs)
            yield step, k, vals, rhs, dU
            U = U + dU


def _solver(pb, vals, nd, pt, restart, precision="fp32"):
    prm = fsi.default_params(2, restart=restart, maxit=2000, flags=fsi.FSI_USE_GRAPHS)
    S = fsi.FSISolver(2, pb.rowptr, pb.colind, vals, pb.offsets, pb.solid_node_coords(), prm)
    S.precond_build(precision)
    S.learned_setup(nd, pt)
    return S


def harvest(cfg, steps=50, newton=3, keep_every=5, nvec=8, restart=40, rtol=1e-10, log=None):
    """Run the trajectory; keep the solvers of every `keep_every`-th time step with
    the r' vectors of their first `nvec` iterations.  Returns (kept, newton_log)."""
    import torch
    pb = fsigen.get_problem(cfg)
    nd, pt = pb.node_map()
    kept, nlog = [], []
    state = {}

    def solve(step, k, vals, rhs):
        S = _solver(pb, vals, nd, pt, restart)
        keep = (step % keep_every) == keep_every - 1
        buf = torch.zeros((nvec, pb.n), dtype=torch.float64, device="cuda") if keep else None
        if keep:
            S.set_harvest(buf, nvec)
        b = torch.from_numpy(rhs).cuda()
        x = torch.zeros_like(b)
        st = S.solve(b, x, rtol=rtol, raise_on_error=False)
        torch.cuda.synchronize()
        rec = {"step": step, "newton": k, "rhs_norm": float(np.linalg.norm(rhs)), "iters": st.iters,
               "relres": st.true_relres, "status": st.status}
        nlog.append(rec)
        if log:
            log(rec)
        if keep:
            S.set_harvest(None)
            m = min(nvec, st.iters) if st.cycles <= 1 else nvec
            R = buf[:m].clone()
            good = [i for i in range(m) if torch.linalg.vector_norm(R[i]).item() > 0]
            if good:
                kept.append((S, R[good], (step, k)))
            else:
                S.close()
        else:
            S.close()
        state["last"] = x
        return x.cpu().numpy()

    for _ in newton_trajectory(cfg, steps, newton, solve):
        pass
    return kept, nlog


def class_scales(kept, offsets, fixed, rtol=1e-10):
    """sigma_in[c] = RMS of r' over free class-c DOFs (all kept residuals);
    sigma_out[c] = RMS of the error e = A^-1 r' (first residual of each kept solver)."""
    import torch
    off = np.asarray(offsets)
    free = torch.from_numpy(~np.asarray(fixed, bool)).cuda()
    sums_in, cnt_in = np.zeros(5), np.zeros(5)
    sums_out, cnt_out = np.zeros(5), np.zeros(5)
    for S, R, _ in kept:
        for i in range(R.shape[0]):
            for c in range(5):
                sl = slice(int(off[c]), int(off[c + 1]))
                v = R[i, sl][free[sl]]
                sums_in[c] += float((v * v).sum())
                cnt_in[c] += v.numel()
        e = torch.zeros_like(R[0])
        S.solve(R[0].contiguous(), e, rtol=rtol, raise_on_error=False)
        torch.cuda.synchronize()
        for c in range(5):
            sl = slice(int(off[c]), int(off[c + 1]))
            v = e[sl][free[sl]]
            sums_out[c] += float((v * v).sum())
            cnt_out[c] += v.numel()
    sig_in = np.sqrt(sums_in / np.maximum(cnt_in, 1))
    sig_out = np.sqrt(sums_out / np.maximum(cnt_out, 1))
    sig_in[~(sig_in > 0)] = 1.0
    sig_out[~(sig_out > 0)] = 1.0
    return sig_in.astype(np.float32), sig_out.astype(np.float32)


def train(kept, sig_in, sig_out, epochs=40, batch=8, lr=1e-3, lr_final=1e-4, seed=0, holdout=1, log=None):
    """AdamW over the kept (solver, r') pairs, cosine-decayed rate from lr to
    lr_final; the last `holdout` solvers are validation only.  Returns (trainer, history)."""
    pairs = [(S, R[i]) for S, R, _ in kept[:len(kept) - holdout] for i in range(R.shape[0])]
    val = [(S, R[i]) for S, R, _ in kept[len(kept) - holdout:] for i in range(R.shape[0])]
    tr = fsi.Trainer(lr=lr, seed=seed, sigma_in=list(sig_in), sigma_out=list(sig_out))
    rng = np.random.default_rng(seed)
    hist = []
    n_upd = max(1, epochs * math.ceil(len(pairs) / batch))
    upd = 0
    for ep in range(epochs):
        order = rng.permutation(len(pairs))
        losses = []
        rate = lr
        for b0 in range(0, len(order), batch):
            rate = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * upd / n_upd))
            S_last = None
            for i in order[b0:b0 + batch]:
                S, r = pairs[i]
                losses.append(tr.step(S, r))
                S_last = S
            tr.update(S_last, rate)
            upd += 1
        rec = {"epoch": ep, "train_loss": float(np.mean(losses)), "lr": rate}
        if val:
            rec["val_loss"] = float(np.mean([tr.loss(S, r) for S, r in val]))
        hist.append(rec)
        if log:
            log(rec)
    return tr, hist


def sweep(S, b, x_exact, taus, log, tag):
    """Solve b with the plain FP32-AMG form and with the learned stage at each
    accept ratio (graphs on, one warm-up solve each); log iterations, seconds,
    accepted corrections and the error against x_exact (when given)."""
    import torch

    def err(x):
        if x_exact is None:
            return None
        return float(torch.linalg.vector_norm(x - x_exact) / torch.linalg.vector_norm(x_exact))

    x0 = torch.zeros_like(b)
    S.set_flags(fsi.FSI_USE_GRAPHS)
    S.solve(b, x0, rtol=1e-8, raise_on_error=False)
    x0.zero_()
    p = S.solve(b, x0, rtol=1e-8, raise_on_error=False)
    log(dict(tag, form="fp32_amg", iters=p.iters, solve_s=p.solve_s, relres=p.true_relres, err_vs_xstar=err(x0)))
    for tau in taus:
        S.set_learned_accept(tau)
        S.set_flags(fsi.FSI_USE_GRAPHS | fsi.FSI_LEARNED)
        x1 = torch.zeros_like(b)
        S.solve(b, x1, rtol=1e-8, raise_on_error=False)
        x1.zero_()
        q = S.solve(b, x1, rtol=1e-8, raise_on_error=False)
        log(dict(tag, form="learned", tau=tau, iters=q.iters, accepted=q.learned_accepted, solve_s=q.solve_s,
                 relres=q.true_relres, err_vs_xstar=err(x1),
                 x_vs_plain=float(torch.linalg.vector_norm(x1 - x0) / torch.linalg.vector_norm(x0))))
    S.set_flags(fsi.FSI_USE_GRAPHS)
    S.set_learned_accept(0.1)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--out", default=DEFAULT_WEIGHTS)
    t.add_argument("--nx", type=int, default=256)
    t.add_argument("--ny", type=int, default=128)
    t.add_argument("--steps", type=int, default=50)
    t.add_argument("--newton", type=int, default=3)
    t.add_argument("--keep-every", type=int, default=5)
    t.add_argument("--nvec", type=int, default=8)
    t.add_argument("--epochs", type=int, default=40)
    t.add_argument("--batch", type=int, default=8)
    t.add_argument("--lr", type=float, default=1e-3)
    t.add_argument("--seed", type=int, default=0)
    e = sub.add_parser("evaluate")
    e.add_argument("--weights", default=DEFAULT_WEIGHTS)
    e.add_argument("--config", default="2d_mid")
    e.add_argument("--states", type=int, default=3)
    e.add_argument("--taus", default="1,0.5,0.3,0.1")
    e.add_argument("--trajectory", type=int, default=0,
                   help="evaluate Newton systems of the last two of this many trajectory steps instead")
    e.add_argument("--nx", type=int, default=256)
    e.add_argument("--ny", type=int, default=128)
    a = ap.parse_args(argv)
    import torch
    torch.cuda.init()

    def log(rec):
        print(json.dumps(rec), flush=True)

    if a.cmd == "train":
        cfg = fsigen.CONFIGS["2d_mid"].with_(name=f"2d_{a.nx}x{a.ny}", n=(a.nx, a.ny))
        pb = fsigen.get_problem(cfg)
        t0 = time.perf_counter()
        kept, nlog = harvest(cfg, a.steps, a.newton, a.keep_every, a.nvec, log=log)
        t1 = time.perf_counter()
        sig_in, sig_out = class_scales(kept, pb.offsets, pb.fixed)
        log({"sigma_in": sig_in.tolist(), "sigma_out": sig_out.tolist(), "kept_solvers": len(kept),
             "vectors": int(sum(R.shape[0] for _, R, _ in kept)), "harvest_s": t1 - t0})
        tr, hist = train(kept, sig_in, sig_out, a.epochs, a.batch, a.lr, seed=a.seed, log=log)
        tr.save(a.out)
        log({"saved": a.out, "train_s": time.perf_counter() - t1})
        return 0
    # evaluate: plain FP32-AMG form against the same form with the learned stage
    taus = [float(v) for v in a.taus.split(",")]
    if a.trajectory:
        # systems of the training trajectory beyond the harvested steps (in distribution)
        cfg = fsigen.CONFIGS["2d_mid"].with_(name=f"2d_{a.nx}x{a.ny}", n=(a.nx, a.ny))
        pb = fsigen.get_problem(cfg)
        nd, pt = pb.node_map()

        def solve(step, k, vals, rhs):
            S = _solver(pb, vals, nd, pt, 100)
            b = torch.from_numpy(rhs).cuda()
            x = torch.zeros_like(b)
            S.solve(b, x, rtol=1e-10, raise_on_error=False)
            if step >= a.trajectory - 2 and k < 2:
                S.learned_load(a.weights)
                sweep(S, b, None, taus, log, {"trajectory_step": step, "newton": k, "mesh": [a.nx, a.ny]})
            S.close()
            return x.cpu().numpy()

        for _ in newton_trajectory(cfg, a.trajectory, 3, solve):
            pass
        return 0
    cfg = fsigen.CONFIGS[a.config]
    pb = fsigen.get_problem(cfg)
    nd, pt = pb.node_map()
    for s in range(a.states):
        sysm = fsigen.make_system(cfg, state_seed=s, rhs_seed=s)
        S = _solver(pb, sysm.vals, nd, pt, 100)
        S.learned_load(a.weights)
        sweep(S, torch.from_numpy(sysm.rhs).cuda(), torch.from_numpy(sysm.x_exact).cuda(), taus, log,
              {"config": a.config, "state": s})
        S.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
