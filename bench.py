#!/usr/bin/env python
"""Benchmark of the Newton-step linear solve: right-preconditioned FGMRES with
the block-LDU preconditioner (Alg. 2) on the 2D 256x128 Q2/Q2/Q1 ALE-FSI
Jacobian (n = 560,517, five seeded linearisation states, rtol 1e-8), FP32-AMG
form (hierarchies and smoothers in FP32 inside FP64 FGMRES), on one GB300.

One step = one fsi_solve of one resident Jacobian (steps cycle over the five
states, each ~0.6 GB of matrices, so no step finds the previous one's data in
L2).  Set-up (fsi_setup + fsi_precond_build) is timed apart.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the same workload instead (bounded sample of FGMRES iterations, scaled to a
full solve).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
LEARNED_WEIGHTS = os.path.join(ROOT, "paper_1801_05648_gb300", "weights", "mlp_fsi2d_256x128.bin")
sys.path.insert(0, ROOT)

METRIC = "Newton-step solve seconds to 1e-8 rel. residual (FP32-AMG/learned vs FP64); GB/s"
WORKLOAD_DESC = {
    "2d_mid": "2D ALE-FSI Jacobian, 256x128 Q2/Q2/Q1 cells on [0,2]x[0,1], solid strip y<0.25, n=560517, "
              "5 seeded states",
    "3d": "3D ALE-FSI Jacobian, 32x16x16 Q2/Q2/Q1 hex cells on [0,2]x[0,1]^2, solid slab z<0.25, n=434247",
    "2d_large": "2D ALE-FSI Jacobian, 1024x512 Q2/Q2/Q1 cells, amplitude 5e-2, n=8926725",
    "2d_tiny": "2D ALE-FSI Jacobian, 16x16 Q2/Q2/Q1 cells, n=4645",
}


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="2d_mid")
    ap.add_argument("--states", type=int, default=5)
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-form timing")
    ap.add_argument("--no-pdl", action="store_true", help="launch without programmatic dependent launch")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graphs", action="store_true")
    ap.add_argument("--spmv-prefetch", type=int, default=None, choices=[0, 1, 2],
                    help="SpMV L2 prefetch mode (fsi_params.spmv_prefetch; default: the library's)")
    ap.add_argument("--kernel-only", choices=["spmv", "solve", "mlp"], default=None,
                    help="small programs for ncu captures: 'spmv' runs the outer SpMV 6 times; 'solve' runs "
                         "one solve of the bench workload inside cudaProfilerStart/Stop")
    ap.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--sample-iters", type=int, default=8)
    ap.add_argument("--full-iters", type=int, default=0)
    return ap.parse_args(argv)


# ------------------------------------------------------------------ oracle timing
def oracle_sample(workload: str, state: int, sample_iters: int, full_iters: int, steps: int = 1):
    """Time the CPU oracle: AMG set-up once, then `steps` FGMRES runs of
    `sample_iters` iterations each; seconds per solve = seconds per iteration
    times `full_iters` (the iteration count of a complete solve)."""
    import fsigen
    import oracle
    cfg = fsigen.CONFIGS[workload].with_(state_seed=state)
    s = fsigen.make_system(cfg)
    prm = oracle.PrecondParams(mass_ratio=8.0 if s.dim == 2 else 20.0)
    t0 = time.perf_counter()
    o = oracle.OracleSolver.from_system(s, params=prm)
    setup = time.perf_counter() - t0
    if full_iters <= 0:
        r = o.solve(s.rhs, tol=1e-8)
        full_iters = r.iters
    per_iter = []
    for _ in range(steps):
        t0 = time.perf_counter()
        r = o.solve(s.rhs, tol=1e-30, maxit=sample_iters, restart=max(sample_iters, 1))
        per_iter.append((time.perf_counter() - t0) / max(r.iters, 1))
    return {"setup_s": setup, "per_iter_s": per_iter, "full_iters": full_iters, "n": s.n}


def blas_threads() -> int:
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k, "").isdigit():
            return int(os.environ[k])
    return os.cpu_count() or 1


def run_cpu_sample_subprocess(workload, sample_iters, full_iters, timeout=600):
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample", "--workload", workload,
           "--sample-iters", str(sample_iters), "--full-iters", str(full_iters)]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=timeout)
    if r.returncode != 0:
        return None, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1]), None


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
            os.unlink(self.path)
        except Exception:
            return None
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ helpers
def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_hash(source_files) -> str:
    h = hashlib.sha256()
    for f in source_files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()


def kernel_traffic(profile_name: str, source_files):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from a
    committed ncu summary under profiles/, read from its 'dram_bytes_per_launch:'
    and 'source_sha256:' lines; None when the kernel sources changed since."""
    path = os.path.join(ROOT, "profiles", profile_name)
    vals = {}
    try:
        for line in open(path):
            if ":" in line and line.split(":", 1)[0].strip() in ("dram_bytes_per_launch", "source_sha256"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
    except OSError:
        return None
    if vals.get("source_sha256") != source_hash(source_files):
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def dist_setup(args=None):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------------ replicas (N > 1)
# The solve does not shard: one Jacobian per GPU.  With N ranks each solves its
# own seeded Jacobians (replicas); the only collectives are the barriers around
# the timed region and the max of the per-rank step time.
def replica_seeds(rank: int, states: int):
    """State seeds of one rank's resident Jacobians (disjoint across ranks)."""
    return [rank * states + k for k in range(states)]


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank float over the process group (value itself at N = 1)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_seconds_per_solve(step_ms_max: float, world: int) -> float:
    """Whole-job seconds per solved Jacobian: each of `world` ranks solves one
    Jacobian per step, the step lasting as long as the slowest rank."""
    return step_ms_max / 1e3 / world


# ------------------------------------------------------------------ our arm
def bench_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    import fsigen
    from paper_1801_05648_gb300 import build as libbuild
    import paper_1801_05648_gb300 as P

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    libbuild.build()
    dev = torch.device("cuda", local)
    bs = torch.cuda.Stream(device=dev)       # every solver runs on this stream
    flags = (0 if args.no_graphs else P.FSI_USE_GRAPHS) | (P.FSI_NO_PDL if args.no_pdl else 0)

    systems, solvers = [], []
    setup_s, build_s = [], []
    for seed in replica_seeds(rank, args.states):
        cfg = fsigen.CONFIGS[args.workload].with_(state_seed=seed)
        s = fsigen.make_system(cfg)
        knobs = {} if args.spmv_prefetch is None else {"spmv_prefetch": args.spmv_prefetch}
        g = P.FSISolver.from_system(s, params=P.default_params(s.dim, mass_ratio=8.0 if s.dim == 2 else 20.0,
                                                               flags=flags, **knobs), stream=bs)
        t0 = time.perf_counter()
        g.precond_build("fp64")
        build_s.append(time.perf_counter() - t0)
        systems.append(s)
        solvers.append(g)
    n = systems[0].n
    rhs = [torch.tensor(s.rhs, device=dev) for s in systems]
    xs = [torch.zeros(n, dtype=torch.float64, device=dev) for _ in systems]
    S = len(systems)

    def run_steps(k0, count, stats):
        for k in range(k0, k0 + count):
            st = solvers[k % S].solve(rhs[k % S], xs[k % S], 1e-8)
            stats.append(st)

    def timed(prec, steps, warmup):
        for g in solvers:
            g.precond_build(prec)
        warm = []
        run_steps(0, warmup, warm)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        st = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(bs):
            e0.record(bs)
        t0 = time.perf_counter()
        run_steps(warmup, steps, st)
        with torch.cuda.stream(bs):
            e1.record(bs)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if world > 1:
            dist.barrier()
        ms = e0.elapsed_time(e1) / steps
        return ms, wall / steps, st

    # FP64 reference form first (comparison key), then the headline form
    other = "fp64" if args.precision == "fp32" else "fp32"
    ms_o, wall_o, st_o = timed(other, max(3, min(args.steps, 10)), args.warmup)
    err_other = None
    if all(s_.x_exact is not None for s_ in systems):
        err_other = max(float(np.linalg.norm(xs[i].cpu().numpy() - systems[i].x_exact) /
                              np.linalg.norm(systems[i].x_exact)) for i in range(S))
    sampler = ClockSampler(local)
    sampler.start()
    ms, wall, st = timed(args.precision, args.steps, args.warmup)
    clocks = sampler.stop()

    # convergence / correctness of every timed solve; error against the manufactured solution
    relres = max(x.true_relres for x in st)
    def err_vs_exact():
        e = []
        for i in range(S):
            if systems[i].x_exact is not None:
                xe = systems[i].x_exact
                e.append(float(np.linalg.norm(xs[i].cpu().numpy() - xe) / np.linalg.norm(xe)))
        return max(e) if e else None
    err_main = err_vs_exact()
    assert all(x.status == 0 for x in st), "a timed solve did not converge"
    iters = [x.iters for x in st]
    launches = sum(x.kernel_launches for x in st)
    bytes_per_solve = statistics.mean(x.iters * (x.operator_bytes + x.precond_bytes) for x in st)

    # ---- end to end through the C ABI with host buffers (H2D rhs, D2H x inside the region)
    host_b = [torch.empty(n, dtype=torch.float64, pin_memory=True) for _ in systems]
    host_x = [torch.empty(n, dtype=torch.float64, pin_memory=True) for _ in systems]
    for hb, s in zip(host_b, systems):
        hb.copy_(torch.from_numpy(s.rhs))
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(bs)
    for k in range(e2e_steps):
        i = k % S
        with torch.cuda.stream(bs):
            rhs[i].copy_(host_b[i], non_blocking=True)
        solvers[i].solve(rhs[i], xs[i], 1e-8)
        with torch.cuda.stream(bs):
            host_x[i].copy_(xs[i], non_blocking=True)
    e1.record(bs)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    for i in range(min(S, e2e_steps)):
        xc = host_x[i].numpy()
        A = systems[i].scipy()
        rr = np.linalg.norm(systems[i].rhs - A @ xc) / np.linalg.norm(systems[i].rhs)
        assert rr <= 1.001e-8, f"end-to-end result fails the residual check ({rr})"

    # ---- learned form: the headline form plus the learned correction stage (2D only;
    # weights trained on the method's own Newton-step solves, default accept ratio)
    learned = None
    if systems[0].dim == 2 and not args.no_learned:
        pb = fsigen.get_problem(systems[0].cfg)
        nd, pt = pb.node_map()
        for g in solvers:
            g.learned_setup(nd, pt)
            g.learned_load(LEARNED_WEIGHTS)
            g.set_flags(flags | P.FSI_LEARNED)
        ms_l, wall_l, st_l = timed(args.precision, max(3, min(args.steps, 10)), args.warmup)
        for g in solvers:
            g.set_flags(flags)
        assert all(x.status == 0 for x in st_l), "a learned-form solve did not converge"
        # the MLP kernel alone (one launch per resident Jacobian in turn)
        reps = 30
        cs = [torch.empty(n, dtype=torch.float64, device=dev) for _ in systems]
        for k in range(S):
            solvers[k].learned_apply(rhs[k], cs[k], sync=False)
        bs.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(bs)
        for k in range(reps):
            solvers[k % S].learned_apply(rhs[k % S], cs[k % S], sync=False)
        e1.record(bs)
        bs.synchronize()
        mlp_s = e0.elapsed_time(e1) / reps / 1e3
        mlp_flops = nd.shape[0] * 2.0 * (53 * 64 + 64 * 64 + 64 * 5)
        fp32_peak = 152 * 128 * 2 * (clocks.get("sm_max_mhz") or 2070) * 1e6 / 1e12
        mlp_traffic = kernel_traffic(f"mlp_apply_{args.workload}.md", ["paper_1801_05648_gb300/csrc/learned.cu",
                                                             "paper_1801_05648_gb300/csrc/learned.cuh"])
        learned = {"form": "FP32-AMG + learned stage" if args.precision == "fp32" else "FP64 + learned stage",
                   "solve_s": ms_l / 1e3, "iters_median": statistics.median([x.iters for x in st_l]),
                   "accepted_total": sum(x.learned_accepted for x in st_l),
                   "accept_ratio": float(P.default_params(2).learned_accept),
                   "err_vs_exact_max": err_vs_exact(),
                   "weights": os.path.relpath(LEARNED_WEIGHTS, ROOT),
                   "roofline_mlp": {"kernel": "k_mlp<MODE_APPLY>: patch gather + 53-64-64-5 MLP (bfloat16 weights, "
                                              "FP32 FMA) + scatter", "bound": "alu",
                                    "achieved": mlp_flops / mlp_s / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                                    "peak_kind": "FP32 FMA: 152 SMs x 128 lanes x 2 FLOP x max SM clock",
                                    "frac": mlp_flops / mlp_s / 1e12 / fp32_peak, "launch_us": mlp_s * 1e6,
                                    "flops_per_launch": mlp_flops, "traffic": mlp_traffic}}

    # ---- roofline of the dominant kernel: the fused FP32 2x2 Chebyshev SpMV step of the
    # V-cycles, on level 0 of the mesh and fluid-velocity hierarchies of every resident
    # Jacobian in turn (10 matrices, ~0.3 GB together: each launch finds the L2 holding
    # the other nine's data, not its own), launched back to back
    targets = [(g, w) for g in solvers for w in ("mesh", "fluid_velocity")]
    for g, w in targets:
        g.smoother_steps(w, 0, 1)
    bs.synchronize()
    rounds = 6
    cheb_bytes = 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # a few ms of work queued ahead, so the timed launches below are all enqueued
    # before the GPU reaches them (the host needs ~10 us per call, about a launch's length)
    targets[0][0].smoother_steps(targets[0][1], 0, 1000)
    e0.record(bs)
    for _ in range(rounds):
        for g, w in targets:
            cheb_bytes += g.smoother_steps(w, 0, 1)
    e1.record(bs)
    bs.synchronize()
    cheb_launches = rounds * len(targets)
    cheb_s = e0.elapsed_time(e1) / 1e3
    cheb_achieved = cheb_bytes / cheb_s / 1e9
    # ---- the outer FP64 operator (secondary), alternating between the resident Jacobians
    reps = 60
    yv = [torch.empty(n, dtype=torch.float64, device=dev) for _ in systems]
    for k in range(5):
        solvers[k % S].apply_operator(xs[k % S], yv[k % S], sync=False)
    bs.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(bs)
    for k in range(reps):
        solvers[k % S].apply_operator(xs[k % S], yv[k % S], sync=False)
    e1.record(bs)
    bs.synchronize()
    spmv_s = e0.elapsed_time(e1) / reps / 1e3
    op_bytes = st[0].operator_bytes
    achieved = op_bytes / spmv_s / 1e9
    peak, peak_kind = measured_peak()
    srcs = ["paper_1801_05648_gb300/csrc/spmv.cuh", "paper_1801_05648_gb300/csrc/spmv.cu"]
    # DRAM bytes per launch from the ncu summary of this workload (null without one)
    traffic = kernel_traffic(f"spmv_outer_fp64_{args.workload}.md", srcs)
    cheb_traffic = kernel_traffic(f"spmv_cheb_fp32_{args.workload}.md", srcs)

    # ---- CPU baseline: the oracle on this host's cores (bounded sample)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        fp64_iters = statistics.median([x.iters for x in (st if args.precision == "fp64" else st_o)])
        res, err = run_cpu_sample_subprocess(args.workload, args.sample_iters, int(fp64_iters))
        if res:
            per_it = statistics.median(res["per_iter_s"])
            cpu = {"value": per_it * res["full_iters"], "unit": "s", "cores": 1, "kind": "oracle",
                   "sample": f"FP64 oracle (numpy/scipy, 1 BLAS thread): AMG set-up ({res['setup_s']:.1f} s, not "
                             f"in value) then {args.sample_iters} FGMRES iterations on the state-0 Jacobian, "
                             f"{per_it:.3f} s/iteration scaled to the {res['full_iters']} iterations of a full "
                             f"FP64 solve",
                   "setup_s": res["setup_s"]}
        else:
            cpu = {"value": None, "unit": "s", "cores": 1, "kind": "oracle", "sample": f"failed: {err}"}

    # ---- max over ranks
    t_step = max_over_ranks(ms, dev)
    value = job_seconds_per_solve(t_step, world)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_step,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "fp32" else "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": WORKLOAD_DESC.get(args.workload, args.workload),
                   "form": "FP32-AMG" if args.precision == "fp32" else "FP64", "rtol": 1e-8, "restart": 100,
                   "states": S, "graphs": not args.no_graphs, "pdl": not args.no_pdl,
                   "spmv_prefetch": int(P.default_params(systems[0].dim, **knobs).spmv_prefetch),
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "l2": "inputs larger than L2: each step solves another resident Jacobian (~0.6 GB of "
                         "matrices each)"},
        "iters": {"median": statistics.median(iters), "min": min(iters), "max": max(iters)},
        "true_relres_max": relres,
        "err_vs_exact_max": err_main,
        "other_form": {"form": other.upper() if other == "fp64" else "FP32-AMG", "solve_s": ms_o / 1e3,
                       "iters_median": statistics.median([x.iters for x in st_o]), "err_vs_exact_max": err_other},
        "learned_form": learned,
        "setup_s": statistics.mean(x.setup_s for x in st[:S]) if st else None,
        "precond_build_s_fp64": statistics.mean(build_s),
        "solve_algorithmic_gbs": bytes_per_solve / (ms / 1e3) / 1e9,
        "e2e": {"value": e2e_ms / 1e3, "unit": "s", "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8},
        "roofline": {"kernel": f"k_bsr_spmv<float,{systems[0].dim},{systems[0].dim},0,EpiCheb>: fused Chebyshev "
                               "step of the FP32 V-cycle (level 0 of the mesh and fluid-velocity hierarchies)",
                     "bound": "hbm", "achieved": cheb_achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": cheb_achieved / peak, "traffic": cheb_traffic,
                     "algorithmic_bytes": cheb_bytes / cheb_launches, "launch_us": cheb_s / cheb_launches * 1e6},
        "roofline_outer_spmv": {"kernel": "k_bsr_spmv<double,2,2,1,EpiAxpby> + <double,1,2,1,EpiAxpby>: outer "
                                          "FP64 operator (vector rows, pressure rows)",
                                "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                "frac": achieved / peak, "traffic": traffic, "algorithmic_bytes": op_bytes,
                                "launch_us": spmv_s * 1e6},
        "cpu_baseline": cpu,
        "clocks": clocks,
        "gpu_launches": launches,
        "wall_ms_per_step": wall * 1e3,
    }
    for g in solvers:
        g.close()
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ reference arm
def bench_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    ref_iters = max(2, min(args.sample_iters, 4))   # keeps --steps K --warmup W within a few minutes
    args.sample_iters = ref_iters
    full = oracle_sample(args.workload, 0, ref_iters, 0, steps=args.warmup + args.steps)
    per = full["per_iter_s"][args.warmup:]
    per_it = statistics.mean(per)
    value = per_it * full["full_iters"]
    cores = blas_threads()
    line = {
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_it * args.sample_iters * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": args.workload, "description": WORKLOAD_DESC.get(args.workload, args.workload),
                   "form": "FP64 oracle", "rtol": 1e-8, "restart": 100},
        "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle",
                         "sample": f"FP64 numpy/scipy oracle: each step runs {args.sample_iters} FGMRES iterations "
                                   f"on the state-0 Jacobian after one AMG set-up ({full['setup_s']:.1f} s, not in "
                                   f"value); seconds per iteration x {full['full_iters']} iterations of the "
                                   f"oracle's own full solve"},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def kernel_only(args):
    """'spmv': one resident Jacobian, 6 applications of the outer operator.
    'solve': set-up and one warm-up solve unprofiled, then one solve of the
    bench form between cudaProfilerStart and cudaProfilerStop."""
    import torch
    import fsigen
    from paper_1801_05648_gb300 import build as libbuild
    import paper_1801_05648_gb300 as P
    libbuild.build()
    s = fsigen.make_system(args.workload)
    if args.kernel_only == "solve":
        g = P.FSISolver.from_system(s, params=P.default_params(s.dim, mass_ratio=8.0 if s.dim == 2 else 20.0,
                                                               flags=0 if args.no_graphs else P.FSI_USE_GRAPHS))
        g.precond_build(args.precision)
        b = torch.tensor(s.rhs, device="cuda")
        x = torch.zeros_like(b)
        g.solve(b, x, 1e-8)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStart()
        st = g.solve(b, x, 1e-8)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
        print(json.dumps({"kernel_only": "solve", "workload": args.workload, "form": args.precision,
                          "iters": st.iters, "kernel_launches": st.kernel_launches, "solve_s": st.solve_s}))
        g.close()
        return
    if args.kernel_only == "mlp":
        # the learned stage's MLP on one resident Jacobian: 6 applications to the rhs
        pb = fsigen.get_problem(s.cfg)
        nd, pt = pb.node_map()
        g = P.FSISolver.from_system(s)
        g.learned_setup(nd, pt)
        g.learned_load(LEARNED_WEIGHTS)
        b = torch.tensor(s.rhs, device="cuda")
        c = torch.empty_like(b)
        for _ in range(6):
            g.learned_apply(b, c, sync=False)
        g.stream.synchronize()
        assert bool(torch.isfinite(c).all())
        print(json.dumps({"kernel_only": "mlp", "workload": args.workload, "nodes": int(nd.shape[0]),
                          "c_norm": float(torch.linalg.vector_norm(c))}))
        g.close()
        return
    g = P.FSISolver.from_system(s)
    x = torch.tensor(s.x_exact if s.x_exact is not None else s.rhs, device="cuda")
    y = torch.empty_like(x)
    for _ in range(6):
        g.apply_operator(x, y, sync=False)
    g.stream.synchronize()
    err = float(torch.linalg.norm(y.cpu() - torch.from_numpy(s.rhs)) / torch.linalg.norm(torch.from_numpy(s.rhs)))
    assert err <= 1e-12, err
    print(json.dumps({"kernel_only": args.kernel_only, "workload": args.workload, "n": s.n, "rel_check": err}))
    g.close()


def main():
    args = parse_args()
    if args.kernel_only:
        kernel_only(args)
        return
    if args.cpu_sample:
        res = oracle_sample(args.workload, 0, args.sample_iters, args.full_iters, steps=2)
        print(json.dumps(res), flush=True)
        return
    if args.impl == "reference":
        os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
        bench_reference(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    if "--impl" in sys.argv and "reference" in sys.argv or "--cpu-sample" in sys.argv:
        for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ.setdefault(k, "1")
    main()
