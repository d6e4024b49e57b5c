"""The quasi-Newton time step of Sec. 6 (paper_1801_05648_gb300.newton): the
stopping rule ||r_k||_inf < 1e-6 ||r_0||_inf, the re-assembly rule (only when
the last iteration reduced ||r||_inf by less than 10), on a 16x16 channel step
from rest with the FSI-2 inflow profile.  CPU tests drive the iteration with a
sparse direct solve; the GPU test with FGMRES and Alg. 2 (FP32-AMG)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import fsigen


def _problem():
    from paper_1801_05648_gb300 import learned
    cfg = fsigen.CONFIGS["2d_tiny"].with_(name="newton16", n=(16, 16))
    pb = fsigen.get_problem(cfg)
    idx, prof = learned.inflow(pb)
    return pb, (idx, prof * learned.ramp(cfg.dt) * 30.0)


def _direct(scale=1.0):
    def factory(pb, vals):
        lu = spla.splu(sp.csc_matrix(sp.csr_matrix((vals, pb.colind, pb.rowptr), shape=(pb.n, pb.n))))
        return lambda rhs, rtol: (scale * lu.solve(rhs), 1)
    return factory


def test_newton_converges_with_one_assembly():
    from paper_1801_05648_gb300 import newton
    pb, bc = _problem()
    U = np.zeros(pb.n)
    r = newton.newton_step(pb, U, U.copy(), _direct(), fixed_values=bc)
    assert r.converged and r.residuals[-1] < 1e-6 * r.residuals[0]
    assert all(b < a for a, b in zip(r.residuals, r.residuals[1:]))
    # each step reduces the residual far more than 10x: the first Jacobian is kept
    assert r.assemblies == 1 and 2 <= r.iterations <= 5
    assert np.allclose(r.U[bc[0]], bc[1])


def test_newton_reassembles_when_the_reduction_is_below_ten():
    from paper_1801_05648_gb300 import newton
    pb, bc = _problem()
    U = np.zeros(pb.n)
    # half steps reduce the residual by about 2 per iteration: re-assemble every time
    r = newton.newton_step(pb, U, U.copy(), _direct(0.5), fixed_values=bc, max_iter=40)
    assert r.converged
    red = [a / b for a, b in zip(r.residuals, r.residuals[1:])]
    assert max(red) < 10.0
    assert r.assemblies == r.iterations


def test_newton_zero_residual():
    from paper_1801_05648_gb300 import newton
    pb, _ = _problem()
    U = np.zeros(pb.n)
    r = newton.newton_step(pb, U, U.copy(), _direct())
    assert r.converged and r.iterations == 0 and r.assemblies == 0


@pytest.mark.gpu
def test_newton_step_on_the_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_05648_gb300 import build, newton
    build.build()
    pb, bc = _problem()
    U = np.zeros(pb.n)
    ref = newton.newton_step(pb, U, U.copy(), _direct(), fixed_values=bc)
    r = newton.newton_step(pb, U, U.copy(), newton.gpu_solver_factory("fp32"), fixed_values=bc)
    assert r.converged and r.residuals[-1] < 1e-6 * r.residuals[0]
    assert r.iterations <= ref.iterations + 1 and r.assemblies <= r.iterations
    assert all(0 < it <= 100 for it in r.linear_iters)
    # velocities agree (pressure components carry the Jacobian's ~1e14 conditioning)
    o = pb.offsets
    v = np.r_[o[1]:o[2], o[3]:o[4]]
    assert np.linalg.norm(r.U[v] - ref.U[v]) <= 1e-3 * np.linalg.norm(ref.U[v])
