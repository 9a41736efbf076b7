"""GPU parity of the topology-optimisation step (Sec. 5) against the oracle.

The oracle runs the same Picard step (filter, direct FEA solve, sensitivities,
OC bisection) on the CPU from the same initial design; compliance and design
agree step by step.  Compliance decreases monotonically over the first steps
(reading Q22), the volume constraint holds to bisection accuracy and the
densities stay within bounds.
"""
import numpy as np
import pytest

import workloads
from oracle import direct, fem, topopt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _mbb(nx, ny, sub):
    cfg = workloads.small_config(nx, ny, sub, bc="mbb")
    return cfg


def test_topopt_steps_match_oracle():
    from paper_1501_06211_gb300 import ddel
    cfg = _mbb(64, 32, 16)
    nx, ny = cfg["ne"]
    s = ddel.Solver(cfg, tol=1e-11, max_it=20000)
    rho = torch.full((nx * ny,), 0.4, dtype=torch.float64, device="cuda")
    rho_phys = torch.zeros_like(rho)
    ts = s.topopt_state(rho, volfrac=0.4, r_min=1.5, move=0.2, rho_phys=rho_phys)
    grid = fem.Grid(2, nx, ny)
    fixed, f = fem.bc_from_spec(grid, cfg["bc"])
    Ke = fem.element_stiffness(2, 1.0, cfg["nu"])
    H = topopt.filter_matrix((nx, ny), 1.5)
    rho_o = np.full(nx * ny, 0.4)

    def solve(fac):
        return direct.solve(fem.assemble(grid, Ke, fac), f, fixed)

    for k in range(10):
        rho_prev = rho.cpu().numpy()
        assert np.abs(rho_prev - rho_o).max() < 1e-7 * (k + 1)
        s.topopt_step(ts)
        rho_o, c_o, u_o, rf_o = topopt.topopt_step(grid, Ke, 1.0, 3.0, H, rho_o, f, solve, 0.4)
        assert np.allclose(rho_phys.cpu().numpy(), rf_o, rtol=1e-12, atol=1e-7 * (k + 1))
        assert abs(ts.compliance - c_o) <= 1e-8 * c_o, (k, ts.compliance, c_o)
        assert abs(ts.volume - 0.4) < 1e-9
    assert ts.iteration == 10
    assert np.abs(rho.cpu().numpy() - rho_o).max() < 1e-6


def test_topopt_compliance_monotone_and_bounds():
    from paper_1501_06211_gb300 import ddel
    cfg = _mbb(128, 64, 16)
    nx, ny = cfg["ne"]
    s = ddel.Solver(cfg, tol=1e-9, max_it=20000)
    rho = torch.full((nx * ny,), 0.4, dtype=torch.float64, device="cuda")
    ts = s.topopt_state(rho, volfrac=0.4)
    cs = []
    for _ in range(25):
        s.topopt_step(ts)
        cs.append(ts.compliance)
        r = rho.cpu().numpy()
        assert r.min() >= 1e-3 - 1e-15 and r.max() <= 1.0 + 1e-15
        assert abs(ts.volume - 0.4) < 1e-9
    cs = np.array(cs)
    assert np.all(cs[1:] <= cs[:-1] * (1 + 1e-6)), cs
    assert cs[-1] < 0.5 * cs[0]
