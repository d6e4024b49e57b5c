"""Write tests/golden/oracle_<workload>_samples.txt: the FP64 oracle's own solve of
a benchmark Jacobian (state 0, rtol 1e-8, restart 100), sampled at seeded indices,
for element-wise parity at sizes whose oracle solve takes minutes.  Calls nothing
but the input generator and the oracle.

    python tests/golden/make_oracle_samples.py 2d_large

File format: comment lines (#) with the workload, n, iterations, true residual and
the 2-norm of the whole solution, then one line per sample "index value" (value
printed with 17 significant digits)."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import fsigen  # noqa: E402
import oracle  # noqa: E402

N_SAMPLES = 4000
# AMG coarse size of the stored solution (the parity test passes the same value)
COARSE_MAX = 500


def main(workload):
    s = fsigen.make_system(fsigen.CONFIGS[workload].with_(state_seed=0))
    o = oracle.OracleSolver.from_system(s, params=oracle.PrecondParams(
        mass_ratio=8.0 if s.dim == 2 else 20.0, amg=oracle.AMGParams(coarse_max=COARSE_MAX)))
    r = o.solve(s.rhs, tol=1e-8)
    idx = np.sort(np.random.default_rng(1234).choice(s.n, N_SAMPLES, replace=False))
    path = os.path.join(HERE, f"oracle_{workload}_samples.txt")
    with open(path, "w") as f:
        f.write(f"# FP64 oracle solve of the {workload} state-0 Jacobian (b = A x*), rtol 1e-8, restart 100\n")
        f.write(f"# n {s.n}\n# iters {r.iters}\n# true_relres {r.true_relres:.17g}\n")
        f.write(f"# norm2 {np.linalg.norm(r.x):.17g}\n")
        for i in idx:
            f.write(f"{int(i)} {r.x[i]:.17g}\n")
    print(path, r.iters, r.true_relres)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "2d_large")
