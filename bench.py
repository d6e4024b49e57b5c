#!/usr/bin/env python
"""Benchmark of the Newton-step linear solve: right-preconditioned FGMRES with
the block-LDU preconditioner (Alg. 2) to ||b - Ax||/||b|| <= 1e-8 on one GB300.

Headline workload (default): the 2D 1024x512 Q2/Q2/Q1 ALE-FSI Jacobian
(n = 8,926,725), FP32-AMG form (hierarchies and smoothers in FP32 inside FP64
FGMRES).  One step = one fsi_solve of the resident Jacobian (~31 GB of matrices:
every solve streams far more than L2 holds).  Set-up (fsi_setup +
fsi_precond_build) is timed apart.  The same line carries the FP64 and learned
forms of the headline workload, the 256x128 (five seeded states) and 32x16x16
workloads as secondary keys, every form's error against the FP64 oracle on the
256x128 Jacobian, the roofline of the dominant kernel and of the outer FP64
operator, and the oracle timed on the host cores (cpu_baseline).

    python bench.py [--gpus N --steps K --warmup W] [--workload W] [--impl reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the same workload instead: one continuing oracle FGMRES run, each step one
iteration, scaled to the oracle's full iteration count.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
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
    "2d_large": "2D ALE-FSI Jacobian, 1024x512 Q2/Q2/Q1 cells on [0,2]x[0,1], solid strip y<0.25, n=8926725, "
                "seeded state of amplitude 1e-2 (at 5e-2 the seed-0 state compresses the solid past the stability "
                "limit of the St. Venant-Kirchhoff law)",
    "2d_mid": "2D ALE-FSI Jacobian, 256x128 Q2/Q2/Q1 cells on [0,2]x[0,1], solid strip y<0.25, n=560517, "
              "5 seeded states",
    "3d": "3D ALE-FSI Jacobian, 32x16x16 Q2/Q2/Q1 hex cells on [0,2]x[0,1]^2, solid slab z<0.25, n=434247",
    "2d_tiny": "2D ALE-FSI Jacobian, 16x16 Q2/Q2/Q1 cells, n=4645",
    "2d_512x256": "2D ALE-FSI Jacobian, 512x256 Q2/Q2/Q1 cells, n=2235141",
    "2d_mid_p1disc": "2D ALE-FSI Jacobian, 256x128 cells with the Q2-Q2-P1disc element (discontinuous linear "
                     "pressure per fluid cell), n=601092",
}
DEFAULT_STATES = {"2d_large": 1, "2d_mid": 5, "3d": 1, "2d_mid_p1disc": 1}


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="2d_large")
    ap.add_argument("--states", type=int, default=0, help="resident Jacobians (0: the workload's default)")
    ap.add_argument("--secondary", default="2d_mid,3d,2d_mid_p1disc",
                    help="comma-separated secondary workloads ('' for none)")
    ap.add_argument("--no-newton", action="store_true", help="skip the timed Newton step")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-form timing")
    ap.add_argument("--no-pdl", action="store_true", help="launch without programmatic dependent launch")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-error", action="store_true", help="skip the error against the oracle")
    ap.add_argument("--no-graphs", action="store_true")
    ap.add_argument("--spmv-prefetch", type=int, default=None, choices=[0, 1, 2],
                    help="SpMV L2 prefetch mode (fsi_params.spmv_prefetch; default: the library's)")
    ap.add_argument("--spmv-unroll", type=int, default=None, choices=[4, 8],
                    help="SpMV blocks in flight per lane (fsi_params.spmv_unroll; default: the library's)")
    ap.add_argument("--spmv-lane-shift", type=int, default=None, choices=[0, 1, 2, 3, 4],
                    help="FP32 SpMV lanes per block row / 2^shift (fsi_params.spmv_lane_shift; default: the library's)")
    ap.add_argument("--coarse-max", type=int, default=None,
                    help="AMG: coarsen until <= this many scalar rows (fsi_params.coarse_max; default: the library's)")
    ap.add_argument("--spmv-order", type=int, default=None, choices=[0, 1],
                    help="length-ordered rows in the outer operator (fsi_params.spmv_order; default: the library's)")
    ap.add_argument("--spmv-stage", type=int, default=None, choices=[0, 1],
                    help="staged 2 x 2 FP32 Chebyshev steps (fsi_params.spmv_stage; default: the library's)")
    ap.add_argument("--kernel-only", choices=["spmv", "solve", "mlp", "cheb"], default=None,
                    help="small programs for ncu captures: 'spmv' runs the outer SpMV 6 times, 'cheb' 6 level-0 "
                         "Chebyshev steps of the mesh hierarchy, 'mlp' 6 learned-stage applications; 'solve' runs "
                         "one solve of the workload inside cudaProfilerStart/Stop")
    ap.add_argument("--sample-iters", type=int, default=2, help="oracle iterations of the cpu_baseline sample")
    # internal: the oracle runs in a child process (no CUDA in it)
    ap.add_argument("--oracle-child", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--child-out", default=None, help=argparse.SUPPRESS)
    return ap.parse_args(argv)


# ------------------------------------------------------------------ host description
def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":", 1)[0].strip() in ("Model name", "Model"):
                v = line.split(":", 1)[1].strip()
                if v and not v.isdigit():
                    return v
    except Exception:
        pass
    return platform.processor() or platform.machine()


def blas_threads() -> int:
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k, "").isdigit():
            return int(os.environ[k])
    return os.cpu_count() or 1


def recorded_oracle_iters(workload: str):
    """The FP64 oracle's own full-solve iteration count (oracle/full_solves.json)."""
    try:
        d = json.load(open(os.path.join(ROOT, "oracle", "full_solves.json")))
        return int(d[workload]["iters"]), d[workload]
    except Exception:
        return None, None


# ------------------------------------------------------------------ oracle legs (child processes)
def oracle_iteration_times(workload: str, state: int, iters: int):
    """Set up the oracle and run one FGMRES solve of `iters` iterations (tol 1e-30,
    restart 100) from x = 0, timing every iteration from one preconditioner call to
    the next; returns (set-up s, per-iteration s, n)."""
    import numpy as np
    import fsigen
    import oracle
    s = fsigen.make_system(fsigen.CONFIGS[workload].with_(state_seed=state))
    t0 = time.perf_counter()
    o = oracle.OracleSolver.from_system(s, params=oracle.PrecondParams(mass_ratio=8.0 if s.dim == 2 else 20.0))
    setup = time.perf_counter() - t0
    stamps = []

    def M(r):
        stamps.append(time.perf_counter())
        return o.P(r)
    t0 = time.perf_counter()
    oracle.fgmres(lambda v: o.A @ v, M, np.asarray(s.rhs, np.float64), tol=1e-30, restart=100, maxit=iters)
    t1 = time.perf_counter()
    stamps.append(t1)
    per = [b - a for a, b in zip(stamps[:-1], stamps[1:])]
    return setup, per, s.n


def oracle_child(args):
    """Runs in a child process with the BLAS thread count fixed by its environment."""
    import numpy as np
    kind, workload = args.oracle_child.split(":")
    out = {"threads": blas_threads(), "cpus": os.cpu_count()}
    if kind == "sample":
        setup, per, n = oracle_iteration_times(workload, 0, args.sample_iters)
        out.update(setup_s=setup, per_iter_s=per, n=n)
    elif kind == "solve":
        # one full oracle solve at rtol 1e-8 (timed) and, with the solutions saved,
        # the reference solve tightened to rtol 1e-12
        import fsigen
        import oracle
        s = fsigen.make_system(fsigen.CONFIGS[workload].with_(state_seed=0))
        t0 = time.perf_counter()
        o = oracle.OracleSolver.from_system(s, params=oracle.PrecondParams(mass_ratio=8.0 if s.dim == 2 else 20.0))
        out["setup_s"] = time.perf_counter() - t0
        r8 = o.solve(s.rhs, tol=1e-8)
        out.update(solve_s=r8.solve_s, iters=r8.iters, true_relres=r8.true_relres, n=s.n)
        if args.child_out:
            r12 = o.solve(s.rhs, tol=1e-12, restart=200)
            out.update(ref_iters=r12.iters, ref_relres=r12.true_relres, ref_solve_s=r12.solve_s)
            np.savez(args.child_out, x8=r8.x, x12=r12.x)
    print(json.dumps(out), flush=True)


def run_oracle_child(spec: str, threads: int | None = None, timeout: int = 1500, out: str | None = None,
                     sample_iters: int = 2):
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    if threads is not None:
        for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
            env[k] = str(threads)
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-child", spec, "--sample-iters", str(sample_iters)]
    if out:
        cmd += ["--child-out", out]
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


def measured_bf16_tflops():
    """Dense bf16 GEMM TFLOP/s (burst) of MEASURED_PEAKS.json, None if absent."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except Exception:
        return None


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


SPMV_SRCS = ["paper_1801_05648_gb300/csrc/spmv.cuh", "paper_1801_05648_gb300/csrc/spmv.cu"]


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
class Workload:
    """Resident Jacobians of one workload on the device, each with its solver context."""

    def __init__(self, name, seeds, flags, knobs, stream, dev):
        import torch
        import fsigen
        import paper_1801_05648_gb300 as P
        self.name = name
        self.systems, self.solvers, self.build_s = [], [], []
        self.flags = flags
        for seed in seeds:
            s = fsigen.make_system(fsigen.CONFIGS[name].with_(state_seed=seed))
            g = P.FSISolver.from_system(s, params=P.default_params(s.dim, mass_ratio=8.0 if s.dim == 2 else 20.0,
                                                                   flags=flags, **knobs), stream=stream)
            t0 = time.perf_counter()
            g.precond_build("fp64")
            self.build_s.append(time.perf_counter() - t0)
            self.systems.append(s)
            self.solvers.append(g)
        self.n = self.systems[0].n
        self.dim = self.systems[0].dim
        self.rhs = [torch.tensor(s.rhs, device=dev) for s in self.systems]
        self.xs = [torch.zeros(self.n, dtype=torch.float64, device=dev) for _ in self.systems]
        self.stream = stream

    def timed(self, prec, steps, warmup, world=1):
        """Warm-up solves, then `steps` solves bracketed by CUDA events on the solver
        stream (and a barrier at N > 1): (ms per solve, wall s per solve, stats)."""
        import torch
        import torch.distributed as dist
        t0 = time.perf_counter()
        for g in self.solvers:
            g.precond_build(prec)
        build = time.perf_counter() - t0
        S = len(self.solvers)
        for k in range(warmup):
            self.solvers[k % S].solve(self.rhs[k % S], self.xs[k % S], 1e-8)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        st = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        t0 = time.perf_counter()
        for k in range(warmup, warmup + steps):
            st.append(self.solvers[k % S].solve(self.rhs[k % S], self.xs[k % S], 1e-8))
        e1.record(self.stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if world > 1:
            dist.barrier()
        assert all(x.status == 0 for x in st), f"a timed {self.name} solve did not converge"
        return e0.elapsed_time(e1) / steps, wall / steps, st, build

    def err_vs_exact(self):
        import numpy as np
        e = []
        for s, x in zip(self.systems, self.xs):
            if s.x_exact is not None:
                e.append(float(np.linalg.norm(x.cpu().numpy() - s.x_exact) / np.linalg.norm(s.x_exact)))
        return max(e) if e else None

    def close(self):
        for g in self.solvers:
            g.close()
        self.solvers = []


def form_summary(ms, st, extra=None):
    import statistics as stt
    d = {"solve_s": ms / 1e3, "iters_median": stt.median([x.iters for x in st]),
         "iters_min": min(x.iters for x in st), "iters_max": max(x.iters for x in st),
         "true_relres_max": max(x.true_relres for x in st),
         "launches_per_solve": stt.mean(x.kernel_launches for x in st),
         "solve_algorithmic_gbs": stt.mean(x.iters * (x.operator_bytes + x.precond_bytes) for x in st) / (ms / 1e3)
         / 1e9}
    if extra:
        d.update(extra)
    return d


def rel(a, b):
    import numpy as np
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


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
    knobs = {k: v for k, v in (("spmv_prefetch", args.spmv_prefetch), ("spmv_unroll", args.spmv_unroll),
                               ("spmv_lane_shift", args.spmv_lane_shift), ("spmv_stage", args.spmv_stage),
                               ("spmv_order", args.spmv_order),
                               ("coarse_max", args.coarse_max))
             if v is not None}
    n_states = args.states or DEFAULT_STATES.get(args.workload, 1)
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count

    # measured FMA rates of this GPU (the pipes that bound the FP64 operator and the FP32 MLP)
    fma64, _ = P.probe_fma_rate(64, iters=8192, reps=5)
    fma32, _ = P.probe_fma_rate(32, iters=131072, reps=5)

    W = Workload(args.workload, replica_seeds(rank, n_states), flags, knobs, bs, dev)
    S = len(W.solvers)
    n = W.n

    # FP64 form first (comparison key), then the headline form
    other = "fp64" if args.precision == "fp32" else "fp32"
    ms_o, wall_o, st_o, _ = W.timed(other, max(3, min(args.steps, 5)), min(args.warmup, 3), world)
    err_other = W.err_vs_exact()
    sampler = ClockSampler(local)
    sampler.start()
    ms, wall, st, build32 = W.timed(args.precision, args.steps, args.warmup, world)
    clocks = sampler.stop()
    err_main = W.err_vs_exact()
    iters = [x.iters for x in st]
    launches = sum(x.kernel_launches for x in st)
    bytes_per_iter = statistics.mean(x.operator_bytes + x.precond_bytes for x in st)

    # ---- end to end through the C ABI with host buffers (H2D rhs, D2H x inside the region)
    host_b = [torch.empty(n, dtype=torch.float64, pin_memory=True) for _ in range(S)]
    host_x = [torch.empty(n, dtype=torch.float64, pin_memory=True) for _ in range(S)]
    for hb, s in zip(host_b, W.systems):
        hb.copy_(torch.from_numpy(s.rhs))
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(bs)
    for k in range(e2e_steps):
        i = k % S
        with torch.cuda.stream(bs):
            W.rhs[i].copy_(host_b[i], non_blocking=True)
        W.solvers[i].solve(W.rhs[i], W.xs[i], 1e-8)
        with torch.cuda.stream(bs):
            host_x[i].copy_(W.xs[i], non_blocking=True)
    e1.record(bs)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    for i in range(min(S, e2e_steps)):
        xc = host_x[i].numpy()
        A = W.systems[i].scipy()
        rr = np.linalg.norm(W.systems[i].rhs - A @ xc) / np.linalg.norm(W.systems[i].rhs)
        assert rr <= 1.001e-8, f"end-to-end result fails the residual check ({rr})"

    # ---- learned form: the headline form plus the learned correction stage (2D only;
    # weights trained on the method's own Newton-step solves, default accept ratio)
    learned = None
    if W.dim == 2 and not args.no_learned:
        pb = fsigen.get_problem(W.systems[0].cfg)
        nd, pt = pb.node_map()
        for g in W.solvers:
            g.learned_setup(nd, pt)
            g.learned_load(LEARNED_WEIGHTS)
            g.set_flags(flags | P.FSI_LEARNED)
        ms_l, wall_l, st_l, _ = W.timed(args.precision, max(3, min(args.steps, 5)), min(args.warmup, 3), world)
        for g in W.solvers:
            g.set_flags(flags)
        reps = 30
        cs = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(S)]

        def time_mlp(unit_flags):
            for g in W.solvers:
                g.set_flags(flags | unit_flags)
            for k in range(S):
                W.solvers[k].learned_apply(W.rhs[k], cs[k], sync=False)
            bs.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(bs)
            for k in range(reps):
                W.solvers[k % S].learned_apply(W.rhs[k % S], cs[k % S], sync=False)
            e1.record(bs)
            bs.synchronize()
            for g in W.solvers:
                g.set_flags(flags)
            return e0.elapsed_time(e1) / reps / 1e3

        mlp_s = time_mlp(0)                          # tcgen05 (the default)
        mlp_cc_s = time_mlp(P.FSI_MLP_CUDA_CORES)    # FP32 FMAs on the CUDA cores
        mlp_flops = nd.shape[0] * 2.0 * (53 * 64 + 64 * 64 + 64 * 5)
        fp32_peak = 2.0 * fma32 / 1e12
        # TF32 dense peak: the measured bf16 GEMM rate x the nominal TF32 / bf16 ratio (1.1 / 2.25)
        bf16_peak = measured_bf16_tflops()
        tf32_peak = bf16_peak * (1.1 / 2.25) if bf16_peak else 2250.0 * (1.1 / 2.25)
        mlp_traffic = kernel_traffic(f"mlp_apply_{args.workload}.md", ["paper_1801_05648_gb300/csrc/mlp_tc.cu",
                                                                     "paper_1801_05648_gb300/csrc/learned.cuh"])
        learned = form_summary(ms_l, st_l, {
            "form": "FP32-AMG + learned stage" if args.precision == "fp32" else "FP64 + learned stage",
            "accepted_total": sum(x.learned_accepted for x in st_l),
            "accept_ratio": float(P.default_params(2).learned_accept), "err_vs_exact_max": W.err_vs_exact(),
            "weights": os.path.relpath(LEARNED_WEIGHTS, ROOT),
            "roofline_mlp": {"kernel": "k_mlp_tc: patch gather + 53-64-64-5 MLP on tcgen05 (kind::tf32, "
                                       "activations as two TF32 terms, bfloat16 weights) + scatter", "bound": "tensor",
                             "achieved": mlp_flops / mlp_s / 1e12, "peak": tf32_peak, "unit": "TFLOP/s",
                             "peak_kind": "measured bf16 GEMM x 1.1/2.25 (nominal TF32 / bf16)" if bf16_peak
                                          else "nominal bf16 x 1.1/2.25",
                             "frac": mlp_flops / mlp_s / 1e12 / tf32_peak, "launch_us": mlp_s * 1e6,
                             "flops_per_launch": mlp_flops, "traffic": mlp_traffic,
                             "cuda_cores": {"kernel": "k_mlp<MODE_APPLY> (FP32 FMA)", "launch_us": mlp_cc_s * 1e6,
                                            "achieved": mlp_flops / mlp_cc_s / 1e12, "peak": fp32_peak,
                                            "peak_kind": "measured FP32 FMA rate x 2 (fsi_probe_fma_rate)",
                                            "frac": mlp_flops / mlp_cc_s / 1e12 / fp32_peak}}})

    # ---- roofline of the dominant kernel: the fused FP32 Chebyshev SpMV step of the
    # V-cycles on level 0 of the mesh and fluid-velocity hierarchies of each resident
    # Jacobian in turn, launched back to back (each launch's matrix is larger than
    # L2, or, with several small Jacobians, the other matrices evict it)
    targets = [(g, w) for g in W.solvers for w in ("mesh", "fluid_velocity")]
    for g, w in targets:
        g.smoother_steps(w, 0, 1)
    bs.synchronize()
    rounds = max(6, 60 // len(targets))
    cheb_bytes = 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # a few ms of work queued ahead, so the timed launches below are all enqueued
    # before the GPU reaches them (the host needs ~10 us per call, about a launch's length)
    targets[0][0].smoother_steps(targets[0][1], 0, 200 if n > 4e6 else 1000)
    e0.record(bs)
    for _ in range(rounds):
        for g, w in targets:
            cheb_bytes += g.smoother_steps(w, 0, 1)
    e1.record(bs)
    bs.synchronize()
    cheb_launches = rounds * len(targets)
    cheb_s = e0.elapsed_time(e1) / 1e3
    cheb_achieved = cheb_bytes / cheb_s / 1e9
    # ---- the outer FP64 operator, alternating between the resident Jacobians
    reps = 30
    yv = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(S)]
    for k in range(3):
        W.solvers[k % S].apply_operator(W.xs[k % S], yv[k % S], sync=False)
    bs.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(bs)
    for k in range(reps):
        W.solvers[k % S].apply_operator(W.xs[k % S], yv[k % S], sync=False)
    e1.record(bs)
    bs.synchronize()
    spmv_s = e0.elapsed_time(e1) / reps / 1e3
    op_bytes = st[0].operator_bytes
    achieved = op_bytes / spmv_s / 1e9
    op_fmas = float(W.systems[0].vals.size)     # one FMA per stored entry of the monolithic operator
    peak, peak_kind = measured_peak()
    traffic = kernel_traffic(f"spmv_outer_fp64_{args.workload}.md", SPMV_SRCS)
    cheb_traffic = kernel_traffic(f"spmv_cheb_fp32_{args.workload}.md", SPMV_SRCS)
    setup_s = statistics.mean(x.setup_s for x in st[:S])
    build64 = statistics.mean(W.build_s)
    W.close()
    del yv
    torch.cuda.empty_cache()

    # ---- secondary workloads: their own resident Jacobians, both forms
    secondary = {}
    err_oracle = None
    names = [w for w in args.secondary.split(",") if w and w != args.workload] if world == 1 else []
    for name in names:
        ns = DEFAULT_STATES.get(name, 1)
        V = Workload(name, list(range(ns)), flags, knobs, bs, dev)
        steps2 = max(ns, 10)
        first0 = (-3) % ns                    # index of the first timed solve of state 0 (3 warm-up solves)
        ms64, _, st64, _ = V.timed("fp64", steps2, 3)
        x64 = V.xs[0].cpu().numpy()
        ms32, _, st32, b32 = V.timed("fp32", steps2, 3)
        x32 = V.xs[0].cpu().numpy()
        entry = {"description": WORKLOAD_DESC.get(name, name), "states": ns,
                 "fp32_amg": form_summary(ms32, st32, {"err_vs_exact_max": V.err_vs_exact()}),
                 "fp64": form_summary(ms64, st64),
                 "setup_s": statistics.mean(x.setup_s for x in st32[:ns]),
                 "precond_build_s_fp64": statistics.mean(V.build_s)}
        xl = None
        if V.dim == 2 and not args.no_learned and V.systems[0].cfg.pressure == "q1":
            pb = fsigen.get_problem(V.systems[0].cfg)
            nd, pt = pb.node_map()
            for g in V.solvers:
                g.learned_setup(nd, pt)
                g.learned_load(LEARNED_WEIGHTS)
                g.set_flags(flags | P.FSI_LEARNED)
            msl, _, stl, _ = V.timed("fp32", steps2, 3)
            xl = V.xs[0].cpu().numpy()
            entry["learned"] = form_summary(msl, stl, {"accepted_total": sum(x.learned_accepted for x in stl)})
        if V.dim == 3 and not args.no_learned and V.systems[0].cfg.pressure == "q1":
            entry["mlp_3d"] = mlp3d_timing(V, bs, fma32)
        secondary[name] = entry
        if name == "2d_mid" and rank == 0 and not args.no_oracle_error:
            err_oracle = {"workload": "2d_mid", "state": 0, "x64": x64, "x32": x32, "xl": xl,
                          "iters64": st64[first0].iters}
        V.close()
        torch.cuda.empty_cache()

    # ---- one quasi-Newton time step (Sec. 6 settings) on the 256x128 channel from rest with
    # the FSI-2 inflow profile: residual and Jacobian assembled on the host (fsigen) against
    # the whole loop on the device (fsi_asm_* + fsi_update_values)
    newton_res = None
    if world == 1 and not args.no_newton:
        newton_res = newton_timing("2d_mid")

    # ---- the oracle on the host cores (child processes: no CUDA there)
    cpu = None
    oracle_err = None
    if rank == 0 and world == 1:
        if err_oracle is not None:
            with tempfile.TemporaryDirectory() as td:
                path = os.path.join(td, "oracle.npz")
                res, err = run_oracle_child("solve:2d_mid", threads=os.cpu_count(), out=path)
                if res:
                    z = np.load(path)
                    x8, x12 = z["x8"], z["x12"]
                    oracle_err = {
                        "workload": "2d_mid", "state": 0,
                        "reference": f"FP64 oracle solve tightened to rtol 1e-12 ({res['ref_iters']} iterations, "
                                     f"true residual {res['ref_relres']:.1e})",
                        "fp64_vs_oracle_same_rtol": rel(err_oracle["x64"], x8),
                        "fp64_iters": err_oracle["iters64"], "oracle_iters": res["iters"],
                        "fp64_vs_reference": rel(err_oracle["x64"], x12),
                        "fp32_amg_vs_reference": rel(err_oracle["x32"], x12),
                        "learned_vs_reference": rel(err_oracle["xl"], x12) if err_oracle["xl"] is not None else None,
                        "oracle_rtol_1e-8_vs_reference": rel(x8, x12),
                        "note": "condition numbers near 1e14-1e16: at a 1e-8 residual the solution is fixed only to "
                                "~1e-3..1e-1 (the oracle's own 1e-8 solve is as far from the reference); forms are "
                                "compared with the oracle at the same tolerance"}
                    oracle_err["full_solve_nproc"] = {"setup_s": res["setup_s"], "solve_s": res["solve_s"],
                                                      "threads": res["threads"]}
                else:
                    oracle_err = {"failed": err}
            res1, _ = run_oracle_child("solve:2d_mid", threads=1)
            if res1 and isinstance(oracle_err, dict):
                oracle_err["full_solve_1thread"] = {"setup_s": res1["setup_s"], "solve_s": res1["solve_s"]}
        if not args.no_cpu_baseline:
            res, err = run_oracle_child(f"sample:{args.workload}", threads=os.cpu_count(),
                                        sample_iters=args.sample_iters)
            full_iters, rec = recorded_oracle_iters(args.workload)
            src = "the oracle's own full solve (oracle/full_solves.json)"
            if full_iters is None:
                full_iters = int(statistics.median([x.iters for x in (st if args.precision == "fp64" else st_o)]))
                src = "the FP64 GPU solve (the oracle's count agrees within one iteration at every size tested)"
            if res:
                per_it = statistics.mean(res["per_iter_s"])
                cpu = {"value": per_it * full_iters, "unit": "s", "cores": res["threads"], "kind": "oracle",
                       "sample": f"FP64 numpy/scipy oracle on the {args.workload} state-0 Jacobian, "
                                 f"{res['threads']} BLAS threads on {res['cpus']} host CPUs ({cpu_model()}): "
                                 f"AMG set-up ({res['setup_s']:.1f} s, not in value), then {len(res['per_iter_s'])} "
                                 f"FGMRES iterations timed one by one ({per_it:.2f} s each) and scaled to the "
                                 f"{full_iters} iterations of {src}",
                       "setup_s": res["setup_s"], "per_iter_s": res["per_iter_s"], "full_iters": full_iters,
                       "host_cpus": res["cpus"], "cpu_model": cpu_model()}
            else:
                cpu = {"value": None, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
                       "sample": f"failed: {err}"}

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
                   "spmv_prefetch": int(P.default_params(W.dim, **knobs).spmv_prefetch),
                   "spmv_unroll": int(P.default_params(W.dim, **knobs).spmv_unroll),
                   "spmv_lane_shift": int(P.default_params(W.dim, **knobs).spmv_lane_shift),
                   "spmv_stage": int(P.default_params(W.dim, **knobs).spmv_stage),
                   "spmv_order": int(P.default_params(W.dim, **knobs).spmv_order),
                   "coarse_max": int(P.default_params(W.dim, **knobs).coarse_max),
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "l2": f"inputs larger than L2: each solve streams {bytes_per_iter / 1e9:.2f} GB of matrices and "
                         f"vectors per FGMRES iteration ({S} resident Jacobian(s); L2 is 0.13 GB)"},
        "iters": {"median": statistics.median(iters), "min": min(iters), "max": max(iters)},
        "true_relres_max": max(x.true_relres for x in st),
        "err_vs_exact_max": err_main,
        "launches_per_solve": launches / len(st),
        "other_form": form_summary(ms_o, st_o, {"form": other.upper() if other == "fp64" else "FP32-AMG",
                                                "err_vs_exact_max": err_other}),
        "learned_form": learned,
        "setup_s": setup_s,
        "precond_build_s_fp64": build64,
        "precond_build_s_fp32": build32 / S,
        "solve_algorithmic_gbs": bytes_per_iter * statistics.mean(iters) / (ms / 1e3) / 1e9,
        "e2e": {"value": e2e_ms / 1e3, "unit": "s", "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8},
        "roofline": {"kernel": f"k_bsr_spmv<float,{W.dim},{W.dim},0,EpiCheb>: fused Chebyshev step of the FP32 "
                               "V-cycle (level 0 of the mesh and fluid-velocity hierarchies)",
                     "bound": "hbm", "achieved": cheb_achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": cheb_achieved / peak, "traffic": cheb_traffic,
                     "algorithmic_bytes": cheb_bytes / cheb_launches, "launch_us": cheb_s / cheb_launches * 1e6},
        "roofline_outer_spmv": {"kernel": f"k_bsr_spmv<double,{W.dim},{W.dim},1,EpiAxpby> + "
                                          f"<double,1,{W.dim},1,EpiAxpby>: outer FP64 operator (vector rows, "
                                          "pressure rows)",
                                "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                "frac": achieved / peak, "traffic": traffic, "algorithmic_bytes": op_bytes,
                                "launch_us": spmv_s * 1e6,
                                "fp64_pipe": {"fmas_per_launch": op_fmas, "achieved_fma_per_s": op_fmas / spmv_s,
                                              "peak_fma_per_s": fma64, "frac": op_fmas / spmv_s / fma64,
                                              "peak_kind": "measured FP64 FMA rate (fsi_probe_fma_rate)"}},
        "measured_fma_rates": {"fp64_fma_per_s": fma64, "fp32_fma_per_s": fma32,
                               "how": "fsi_probe_fma_rate: 8 independent FMA chains per thread, 8 CTAs of 256 "
                                      "threads per SM, best of 5 launches"},
        "secondary": secondary,
        "newton_step": newton_res,
        "err_vs_oracle": oracle_err,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "gpu_launches": launches,
        "wall_ms_per_step": wall * 1e3,
    }
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def bf16_words(w):
    """float32 -> bfloat16 bit patterns, round to nearest even."""
    import numpy as np
    u = np.ascontiguousarray(w, np.float32).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)


def mlp3d_timing(V, bs, fma32, reps: int = 20):
    """The learned stage's MLP on a 3D mesh (3x3x3 patch, 201-64-64-7, CUDA cores):
    seeded random weights (no 3D weights are trained), CUDA events over reps
    applications to the rhs of the first resident Jacobian."""
    import numpy as np
    import torch
    import fsigen
    import paper_1801_05648_gb300 as P
    g = V.solvers[0]
    nd, pt = fsigen.get_problem(V.systems[0].cfg).node_map()
    g.learned_setup(nd, pt)
    w = np.random.default_rng(2024).standard_normal(P.mlp_params(3)) * 0.1
    g.learned_set_weights(np.ones(5, np.float32), np.full(5, 1e-3, np.float32), bf16_words(w))
    b = V.rhs[0]
    c = torch.empty_like(b)
    for _ in range(3):
        g.learned_apply(b, c, sync=False)
    bs.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(bs)
    for _ in range(reps):
        g.learned_apply(b, c, sync=False)
    e1.record(bs)
    bs.synchronize()
    g.check_device_errors()
    t = e0.elapsed_time(e1) / reps / 1e3
    flops = nd.shape[0] * 2.0 * (201 * 64 + 64 * 64 + 64 * 7)
    peak = 2.0 * fma32 / 1e12
    return {"kernel": "k_mlp<3, MODE_APPLY>: 3x3x3 patch gather + 201-64-64-7 MLP (FP32 FMA) + scatter",
            "nodes": int(nd.shape[0]), "launch_us": t * 1e6, "flops_per_launch": flops, "bound": "alu",
            "achieved": flops / t / 1e12, "peak": peak, "unit": "TFLOP/s",
            "peak_kind": "measured FP32 FMA rate x 2 (fsi_probe_fma_rate)", "frac": flops / t / 1e12 / peak,
            "weights": "seeded random (numpy seed 2024, N(0, 0.1^2)); no trained 3D weights"}


def newton_timing(name: str):
    """Wall seconds of one quasi-Newton time step (linear solves FP32-AMG to 1e-3,
    stop at 1e-6 of the initial residual) with host and with device assembly."""
    import numpy as np
    import torch
    import fsigen
    import paper_1801_05648_gb300 as P
    from paper_1801_05648_gb300 import learned, newton
    cfg = fsigen.CONFIGS[name]
    pb = fsigen.get_problem(cfg)
    idx, prof = learned.inflow(pb)
    bc = (idx, prof * learned.ramp(cfg.dt))
    U = np.zeros(pb.n)
    out = {"workload": name, "case": "first step of the channel from rest, FSI-2 inflow profile x ramp(dt)"}
    newton.newton_step_device(pb, U, U.copy(), "fp32", fixed_values=bc)          # warm-up (builds, graphs)
    t0 = time.perf_counter()
    host = newton.newton_step(pb, U, U.copy(), newton.gpu_solver_factory("fp32"), fixed_values=bc)
    host_s = time.perf_counter() - t0
    dev = newton.newton_step_device(pb, U, U.copy(), "fp32", fixed_values=bc)
    for k, r, sec in (("host_assembly", host, host_s), ("device_assembly", dev, dev.seconds)):
        out[k] = {"seconds": sec, "iterations": r.iterations, "assemblies": r.assemblies,
                  "linear_iters": r.linear_iters, "residual_reduction": r.residuals[-1] / r.residuals[0],
                  "converged": bool(r.converged)}
    # the assembly kernels alone at the converged state, against the host assembly
    asm = P.FSIAssembler.from_problem(pb)
    Ud = torch.tensor(dev.U, device="cuda")
    R = torch.empty_like(Ud)
    vals = torch.empty(int(pb.rowptr[-1]), dtype=torch.float64, device="cuda")
    asm.residual(Ud, Ud, R)
    asm.jacobian(Ud, Ud, vals)
    reps = 5
    t0 = time.perf_counter()
    for _ in range(reps):
        asm.residual(Ud, Ud, R)
    out["device_residual_s"] = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        asm.jacobian(Ud, Ud, vals)
    out["device_jacobian_s"] = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    pb.jacobian(dev.U, dev.U)
    out["host_jacobian_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    pb.residual(dev.U, dev.U)
    out["host_residual_s"] = time.perf_counter() - t0
    asm.close()
    return out


# ------------------------------------------------------------------ reference arm
def bench_reference(args):
    """The FP64 oracle on the host cores: AMG set-up once (reported, not in the
    value), then one continuing FGMRES run of W + K iterations from x = 0 whose
    iterations are timed one by one; the first W are warm-up.  value = the mean of
    the K timed iterations x the oracle's full-solve iteration count (seconds per
    solve, the metric's unit); ms_per_step is that per-solve time in ms."""
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    setup, per, n = oracle_iteration_times(args.workload, 0, args.warmup + args.steps)
    timed = per[args.warmup:] or per
    per_it = statistics.mean(timed)
    full_iters, _ = recorded_oracle_iters(args.workload)
    src = "the oracle's own full solve (oracle/full_solves.json)"
    if full_iters is None:
        import fsigen
        import oracle
        s = fsigen.make_system(fsigen.CONFIGS[args.workload])
        o = oracle.OracleSolver.from_system(s, params=oracle.PrecondParams(mass_ratio=8.0 if s.dim == 2 else 20.0))
        full_iters = o.solve(s.rhs, tol=1e-8).iters
        src = "the oracle's own full solve (run here)"
    value = per_it * full_iters
    cores = blas_threads()
    line = {
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": args.workload, "description": WORKLOAD_DESC.get(args.workload, args.workload),
                   "form": "FP64 oracle", "rtol": 1e-8, "restart": 100},
        "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle",
                         "sample": f"FP64 numpy/scipy oracle, {cores} BLAS threads on {os.cpu_count()} host CPUs "
                                   f"({cpu_model()}), {args.workload} state-0 Jacobian: AMG set-up ({setup:.1f} s, "
                                   f"not in value), then one FGMRES run whose iterations are timed one by one "
                                   f"({args.warmup} warm-up, {len(timed)} timed, {per_it:.3f} s each) and scaled to "
                                   f"the {full_iters} iterations of {src}; ms_per_step is the resulting "
                                   f"per-solve time",
                         "setup_s": setup, "per_iter_s": timed, "full_iters": full_iters},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def kernel_only(args):
    """'spmv': one resident Jacobian, 6 applications of the outer operator.
    'cheb': 6 fused Chebyshev steps on level 0 of the mesh hierarchy (FP32-AMG).
    'mlp': 6 learned-stage applications.  'solve': set-up and one warm-up solve
    unprofiled, then one solve of the bench form between cudaProfilerStart and
    cudaProfilerStop."""
    import numpy as np
    import torch
    import fsigen
    from paper_1801_05648_gb300 import build as libbuild
    import paper_1801_05648_gb300 as P
    libbuild.build()
    s = fsigen.make_system(args.workload)
    mr = 8.0 if s.dim == 2 else 20.0
    if args.kernel_only == "solve":
        g = P.FSISolver.from_system(s, params=P.default_params(s.dim, mass_ratio=mr,
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
    if args.kernel_only == "cheb":
        g = P.FSISolver.from_system(s, params=P.default_params(s.dim, mass_ratio=mr))
        g.precond_build("fp32")
        b = g.smoother_steps("mesh", 0, 6)
        g.stream.synchronize()
        print(json.dumps({"kernel_only": "cheb", "workload": args.workload, "bytes_per_step": b}))
        g.close()
        return
    if args.kernel_only == "mlp":
        # the learned stage's MLP on one resident Jacobian: 6 applications to the rhs
        pb = fsigen.get_problem(s.cfg)
        nd, pt = pb.node_map()
        g = P.FSISolver.from_system(s)
        g.learned_setup(nd, pt)
        if s.dim == 2:
            g.learned_load(LEARNED_WEIGHTS)
        else:
            w = np.random.default_rng(2024).standard_normal(P.mlp_params(3)) * 0.1
            g.learned_set_weights(np.ones(5, np.float32), np.full(5, 1e-3, np.float32), bf16_words(w))
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
    if args.oracle_child:
        oracle_child(args)
        return
    if args.kernel_only:
        kernel_only(args)
        return
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
