"""Bounded waits inside kernels give up, report, and leave the context usable.

Failures are made on the host (fsi_debug_inject), never by faulting the GPU: the
FSI_GRID_COARSE kernel's grid barrier is told to wait for one CTA more than its
launch has, and the tensor-core MLP skips the commit of its first layer's MMAs to
the mbarrier it then waits on.  Each wait gives up after its bound (about a second),
sets the kernel's error flag and lets the kernel end.  fsi_check_device_errors then
reports FSI_ECUDA and clears the flags, and with the injection off the same context
solves exactly as before."""
import numpy as np
import pytest

import fsigen
from oracle import learned as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_05648_gb300 import build
    build.build()
    return torch


def test_coarse_grid_barrier_timeout_is_reported(torch_cuda):
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    s = fsigen.make_system(fsigen.CONFIGS["2d_tiny"])
    g = P.FSISolver.from_system(s, params=P.default_params(2, flags=P.FSI_GRID_COARSE))
    try:
        g.precond_build("fp32")
        b = torch.tensor(s.rhs, device="cuda")
        x0 = torch.zeros_like(b)
        st0 = g.solve(b, x0, 1e-8)
        assert st0.status == 0
        g.check_device_errors()                       # nothing pending
        g.debug_inject(P.FSI_INJECT_COARSE_BARRIER)
        y = torch.empty_like(b)
        g.apply_block("precond", b, y)                # V-cycles through the coarse kernel
        with pytest.raises(P.FSIError) as e:
            g.check_device_errors()
        assert e.value.code == P.FSI_ECUDA and "grid barrier" in str(e.value)
        g.debug_inject(0)
        g.check_device_errors()                       # the flags were cleared
        x = torch.zeros_like(b)
        st = g.solve(b, x, 1e-8)
        assert st.status == 0 and st.iters == st0.iters and torch.equal(x, x0)
    finally:
        g.close()


def test_tensor_core_mlp_wait_timeout_is_reported(torch_cuda):
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    s = fsigen.make_system(fsigen.CONFIGS["2d_tiny"])
    nd, pt = fsigen.get_problem(s.cfg).node_map()
    g = P.FSISolver.from_system(s, params=P.default_params(2))
    try:
        g.learned_setup(nd, pt)
        bits = L.bf16_bits(np.random.default_rng(5).standard_normal(L.N_PARAMS) * 0.3)
        g.learned_set_weights(np.ones(5, np.float32), np.ones(5, np.float32), bits)
        r = torch.tensor(np.random.default_rng(6).standard_normal(s.n), device="cuda")
        c0 = torch.empty_like(r)
        g.learned_apply(r, c0)
        g.check_device_errors()
        g.debug_inject(P.FSI_INJECT_MLP_COMMIT)
        c = torch.empty_like(r)
        g.learned_apply(r, c)
        with pytest.raises(P.FSIError) as e:
            g.check_device_errors()
        assert e.value.code == P.FSI_ECUDA and "tensor-core MLP" in str(e.value)
        g.debug_inject(0)
        g.check_device_errors()
        c1 = torch.empty_like(r)
        g.learned_apply(r, c1)
        g.check_device_errors()
        assert torch.equal(c1, c0)
    finally:
        g.close()


def test_debug_inject_rejects_unknown_bits(torch_cuda):
    torch = torch_cuda
    import paper_1801_05648_gb300 as P
    s = fsigen.make_system(fsigen.CONFIGS["2d_tiny"])
    g = P.FSISolver.from_system(s, params=P.default_params(2))
    try:
        with pytest.raises(P.FSIError) as e:
            g.debug_inject(4)
        assert e.value.code == P.FSI_EINVAL
    finally:
        g.close()
