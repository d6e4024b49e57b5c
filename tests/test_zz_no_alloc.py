"""fsi_mass_solve_noalloc: the solid-mass solve for callers that cannot allocate
device memory when they call (stream capture, foreign allocators).  It must give
the same result as fsi_apply_block(ctx, 4, ...) in FP64, the solve it mirrors, on
consecutive calls that reuse its static scratch, whatever precision the context
was built in (the entry point always solves in FP64).  Kept in a file of its own
so that pytest collects it last."""
import numpy as np
import pytest

import fsigen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mass_solve_noalloc_matches_apply_block(precision):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_05648_gb300 import build
    build.build()
    import paper_1801_05648_gb300 as P
    s = fsigen.make_system(fsigen.CONFIGS["2d_tiny"].with_(name="noalloc", n=(64, 32)))
    g = P.FSISolver.from_system(s)
    g.precond_build("fp64")
    n_su = int(s.offsets[3] - s.offsets[2])
    rng = np.random.default_rng(9)
    rs = [torch.tensor(rng.standard_normal(n_su), device="cuda") for _ in range(2)]
    refs = []
    for r in rs:                                 # FP64 references from the block inverse it mirrors
        ref = torch.zeros_like(r)
        g.apply_block("solid_mass", r, ref)
        refs.append(ref)
    if precision == "fp32":
        g.precond_build("fp32")                  # the FP64 hierarchy stays; apply_block now runs in FP32
    for call, (r, ref) in enumerate(zip(rs, refs)):   # two calls in a row share the scratch
        out = torch.full_like(r, np.nan)
        g.mass_solve_noalloc(r, out)
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= 1e-11 * np.linalg.norm(b), (precision, call)
    g.close()
