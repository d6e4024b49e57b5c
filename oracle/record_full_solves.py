"""Record full FP64 oracle solves of the benchmark workloads: iterations, restart
cycles, set-up and solve seconds, host and thread count.  The bench's CPU
baseline times a bounded sample of oracle iterations on the large workload and
scales it by the iteration count recorded here (a full oracle solve of the
8.9M-DOF Jacobian takes minutes).  Test infrastructure only; run as

    python -m oracle.record_full_solves [workload ...]

which writes oracle/full_solves.json (calls nothing but fsigen and oracle)."""
from __future__ import annotations

import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "full_solves.json")


def record(workload: str, state: int = 0) -> dict:
    import fsigen
    from .precond import PrecondParams
    from .solve import OracleSolver
    t0 = time.perf_counter()
    s = fsigen.make_system(fsigen.CONFIGS[workload].with_(state_seed=state))
    gen = time.perf_counter() - t0
    o = OracleSolver.from_system(s, params=PrecondParams(mass_ratio=8.0 if s.dim == 2 else 20.0))
    r = o.solve(s.rhs, tol=1e-8)
    return {"workload": workload, "state": state, "n": s.n, "iters": r.iters, "cycles": r.cycles,
            "converged": bool(r.converged), "true_relres": r.true_relres, "setup_s": o.setup_s,
            "solve_s": r.solve_s, "generate_s": gen, "machine": platform.machine(),
            "cpus": os.cpu_count(), "blas_threads": os.environ.get("OPENBLAS_NUM_THREADS")}


def main(argv):
    names = argv or ["2d_mid", "3d", "2d_large"]
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for w in names:
        data[w] = record(w)
        print(json.dumps(data[w]), flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:])
