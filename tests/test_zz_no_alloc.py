"""The residual check that allocates nothing, against the context's entry point
and against the oracle's assembled K(rho).

Callers that cannot allocate device memory (an allocator that forbids
cudaMalloc, or a component that only receives device buffers) use
ddel_residual_norm_noalloc, whose scratch is a fixed device array inside the
library.  This file runs last (pytest collects it after the others) and passes
both alone in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

import workloads
from oracle import fem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_residual_matches_context_entry_point():
    from paper_1501_06211_gb300 import ddel
    cfg = workloads.small_config(128, 64, 16, seed=11)
    rho = workloads.density(cfg)
    s = ddel.Solver(cfg, tol=1e-8)
    s.assemble(rho)
    s.factor()
    nx, ny = cfg["ne"]
    plan = ddel.Plan(cfg)
    Ke = torch.as_tensor(plan.element_matrix().ravel(), device="cuda")
    factors = torch.as_tensor(cfg["E"] * rho ** cfg["p"], device="cuda")
    fixed = torch.as_tensor(s.fixed_mask().astype(np.uint8), device="cuda")
    f = torch.as_tensor(s.load_vector(), device="cuda")
    u = torch.zeros_like(f)
    s.solve(f, u)
    grid = fem.Grid(2, nx, ny)
    K_or = fem.assemble(grid, fem.element_stiffness(2, 1.0, cfg["nu"]),
                        fem.element_factors(rho, cfg["E"], cfg["p"])).tocsr()
    # a second, unconverged displacement so that the two calls differ
    u2 = u * 0.5 + 1e-3 * torch.randn_like(u)
    for uu in (u, u2):  # two calls in a row
        code, rn_ref, fn_ref = ddel.ddel_residual_norm(s.h, f, uu)
        assert code == 0
        norms = torch.zeros(2, dtype=torch.float64, device="cuda")
        r = torch.zeros_like(f)
        code = ddel.ddel_residual_norm_noalloc(2, nx, ny, 0, Ke, factors, fixed, f, uu, r, norms)
        assert code == 0
        torch.cuda.synchronize()
        rn, fn = norms.tolist()
        # rounding of K u is of order eps ||K|| ||u|| ~ eps ||f||; the element
        # factors here come from NumPy's pow, the context's from CUDA's, so the
        # two residuals agree to that scale (the converged one is a 1e-9
        # cancellation of f - K u)
        assert abs(rn - rn_ref) <= 1e-12 * fn_ref
        assert abs(fn - fn_ref) <= 1e-14 * fn_ref
        # the residual vector itself: f - K u on the free DOFs
        Ku = torch.zeros_like(f)
        assert ddel.ddel_apply_K(s.h, uu, Ku) == 0
        expect = torch.where(fixed.bool(), torch.zeros_like(f), f - Ku)
        torch.cuda.synchronize()
        assert float((r - expect).abs().max()) <= 1e-12 * float(f.abs().max())
        # and against the oracle's own residual: its assembled K(rho) (3x3
        # Gauss element matrix, eq. NumberTen factors) on the same u
        un = uu.cpu().numpy()
        fn_h = f.cpu().numpy()
        fx = fixed.cpu().numpy().astype(bool)
        r_or = fn_h - K_or @ np.where(fx, 0.0, un)
        r_or[fx] = 0.0
        assert np.abs(r.cpu().numpy() - r_or).max() <= 1e-12 * np.abs(fn_h).max()
        assert abs(rn - np.linalg.norm(r_or)) <= 1e-12 * np.linalg.norm(fn_h[~fx])
        assert abs(fn - np.linalg.norm(fn_h[~fx])) <= 1e-14 * fn


def test_noalloc_rejects_oversized_grid():
    from paper_1501_06211_gb300 import ddel
    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    # 2048 x 1024 elements: 2,100,225 nodes, beyond the 1,048,576-node scratch limit
    code = ddel.ddel_residual_norm_noalloc(2, 2048, 1024, 0, d, d, None, d, d, None, d)
    assert code == ddel.DDEL_EINVAL
