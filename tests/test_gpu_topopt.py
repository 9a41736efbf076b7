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


def test_checkpoint_resume_repeats_the_run_bitwise(tmp_path):
    from paper_1501_06211_gb300 import ddel
    cfg = _mbb(64, 32, 16)
    ne = int(np.prod(cfg["ne"]))

    def run(s, ts, k):
        out = []
        for _ in range(k):
            s.topopt_step(ts)
            out.append(ts.compliance)
        return out

    s = ddel.Solver(cfg, tol=1e-9, max_it=20000)
    rho = torch.full((ne,), 0.4, dtype=torch.float64, device="cuda")
    ts = s.topopt_state(rho, volfrac=0.4)
    run(s, ts, 4)
    path = str(tmp_path / "mbb.ckp")
    s.checkpoint_save(ts, path)
    after = run(s, ts, 4)
    rho_end = rho.cpu().numpy()
    # a fresh context resumes from the file
    s2 = ddel.Solver(cfg, tol=1e-9, max_it=20000)
    rho2 = torch.zeros(ne, dtype=torch.float64, device="cuda")
    ts2 = s2.topopt_state(rho2, volfrac=0.1, r_min=3.0, move=0.5)
    s2.checkpoint_load(ts2, path)
    assert ts2.iteration == 4 and ts2.volfrac == 0.4 and ts2.r_min == 1.5 and ts2.move == 0.2
    assert run(s2, ts2, 4) == after
    assert np.array_equal(rho2.cpu().numpy(), rho_end) and ts2.iteration == 8
    # corrupted, truncated and foreign files are refused
    raw = open(path, "rb").read()
    bad = bytearray(raw)
    bad[200] ^= 1
    open(path + ".bad", "wb").write(bytes(bad))
    open(path + ".short", "wb").write(raw[:-9])
    for p in (path + ".bad", path + ".short", str(tmp_path / "missing.ckp")):
        assert ddel.ddel_checkpoint_load(s2.h, ts2, p) == ddel.DDEL_EINVAL
    other = ddel.Solver(dict(cfg, nu=0.25), tol=1e-9)
    rho3 = torch.zeros(ne, dtype=torch.float64, device="cuda")
    assert ddel.ddel_checkpoint_load(other.h, other.topopt_state(rho3, 0.4), path) == ddel.DDEL_EINVAL


def test_solution_scales_exactly_with_load_and_modulus():
    # u(alpha f) = alpha u(f) and u for E*beta = u / beta (linear elasticity);
    # with powers of two (square roots of 4 included) every rounding scales too
    from paper_1501_06211_gb300 import ddel
    cfg = workloads.small_config(64, 32, 16, seed=2)
    rho = workloads.density(cfg)
    s = ddel.Solver(cfg, tol=1e-10, max_it=20000)
    s.assemble(rho)
    s.factor()
    f = s.load_vector()
    u1, _ = s.solve(f)
    u2, _ = s.solve(4.0 * f)  # a power of two: the scaled solve is exact in floating point
    assert np.array_equal(u2, 4.0 * u1)
    s4 = ddel.Solver(dict(cfg, E=4.0), tol=1e-10, max_it=20000)
    s4.assemble(rho)
    s4.factor()
    u4, _ = s4.solve(f)
    assert np.array_equal(u4 * 4.0, u1)
