"""Tile shapes of the explicit Schur apply, native FP64 and double-float (1, 2
or 4 CTAs per subdomain, ddel_options.schur_split) against the oracle's Schur
complement (eq. 3MatSplit) and against each other, on rings of 64, 128 and
256; whole solves keep the FP64 bar with every shape."""
import numpy as np
import pytest

import workloads
from oracle import dd, direct, fem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "ring64": workloads.small_config(64, 32, 8, seed=4),
    "ring128": workloads.small_config(128, 64, 16, seed=11),
    "ring256": workloads.small_config(128, 64, 32, seed=3),
}


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("mode", [1, 2], ids=["fp64", "double_float"])
@pytest.mark.parametrize("name", list(CASES))
def test_explicit_split_shapes(name, mode):
    from paper_1501_06211_gb300 import ddel
    cfg = CASES[name]
    grid = fem.Grid(2, *cfg["ne"])
    fixed, f = fem.bc_from_spec(grid, cfg["bc"])
    rho = workloads.density(cfg)
    dec, K, dds = dd.build(grid, cfg["sub"], fixed, fem.element_stiffness(2, 1.0, cfg["nu"]),
                           fem.element_factors(rho, cfg["E"], cfg["p"]))
    u_ref = direct.solve(K, f, fixed)
    ys = {}
    for split in (1, 2, 4):
        s = ddel.Solver(cfg, schur_mode=mode, schur_split=split, tol=1e-10, max_it=20000)
        s.assemble(rho)
        s.factor()
        gd = s.gamma_dofs()
        x = np.random.default_rng(7).standard_normal(len(gd))
        y = torch.zeros(len(gd), dtype=torch.float64, device="cuda")
        assert ddel.ddel_schur_apply(s.h, torch.as_tensor(x, device="cuda"), y) == 0
        ys[split] = y.cpu().numpy()
        pos = {int(v): k for k, v in enumerate(dec.gamma_dofs)}
        perm = np.array([pos[int(v)] for v in gd])
        xo = np.zeros(len(gd))
        xo[perm] = x
        assert rel(ys[split], dds.schur_apply(xo)[perm]) < 1e-10, split
        u, st = s.solve(check=False)
        assert st.relres <= 1e-9, (split, st.as_dict())
        assert rel(u, u_ref) <= 1e-8, (split, st.as_dict())
        s.close()
    # the same products in another grouping of the row sums: equal to the
    # rounding of the arithmetic (FP64; double-float, about 48 bits)
    tol = 1e-13 if mode == 1 else 1e-12
    assert rel(ys[1], ys[2]) < tol and rel(ys[4], ys[2]) < tol
