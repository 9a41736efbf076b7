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


@pytest.mark.parametrize("adaptive", [False, True], ids=["fixed_tol", "adaptive_tol"])
def test_checkpoint_resume_repeats_the_run_bitwise(tmp_path, adaptive):
    from paper_1501_06211_gb300 import ddel
    cfg = _mbb(64, 32, 16)
    ne = int(np.prod(cfg["ne"]))
    eta = 0.1 if adaptive else 0.0

    def run(s, ts, k):
        out = []
        for _ in range(k):
            s.topopt_step(ts)
            out.append(ts.compliance)
        return out

    s = ddel.Solver(cfg, tol=1e-9, max_it=20000)
    rho = torch.full((ne,), 0.4, dtype=torch.float64, device="cuda")
    ts = s.topopt_state(rho, volfrac=0.4, tol_eta=eta, tol_max=1e-4)
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
    assert ts2.tol_eta == eta and ts2.tol_max == 1e-4
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


def _fnv1a(data, h=1469598103934665603):
    for b in data:
        h = ((h ^ b) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def test_checkpoint_version1_file_loads(tmp_path):
    # a file of the first format (header without the adaptive-tolerance
    # fields, 144 bytes) still loads; compliance_prev = compliance
    import struct
    from paper_1501_06211_gb300 import ddel
    cfg = _mbb(64, 32, 16)
    ne = int(np.prod(cfg["ne"]))
    s = ddel.Solver(cfg, tol=1e-9, max_it=20000)
    rho = torch.full((ne,), 0.4, dtype=torch.float64, device="cuda")
    ts = s.topopt_state(rho, volfrac=0.4)
    s.topopt_step(ts)
    path = str(tmp_path / "v2.ckp")
    s.checkpoint_save(ts, path)
    raw = open(path, "rb").read()
    assert len(raw) == 168 + 8 * ne + 8
    h1 = bytearray(raw[:144])
    h1[8:12] = struct.pack("<I", 1)
    body = bytes(h1) + raw[168:168 + 8 * ne]
    open(str(tmp_path / "v1.ckp"), "wb").write(body + struct.pack("<Q", _fnv1a(body)))
    rho2 = torch.zeros(ne, dtype=torch.float64, device="cuda")
    ts2 = s.topopt_state(rho2, volfrac=0.4)
    s.checkpoint_load(ts2, str(tmp_path / "v1.ckp"))
    assert ts2.iteration == 1 and ts2.compliance == ts.compliance == ts2.compliance_prev
    assert torch.equal(rho2, rho)


def test_adaptive_tolerance_matches_rule_and_saves_iterations():
    # Sec. 5 / Table 3 (reading Q23): the library's per-step tolerance is the
    # oracle's rule applied to the compliances it returned, bit for bit; the
    # run reaches the fixed-tolerance design's compliance with fewer PCG
    # iterations
    from paper_1501_06211_gb300 import ddel
    cfg = _mbb(128, 64, 16)
    ne = int(np.prod(cfg["ne"]))

    def run(eta, steps=60):
        s = ddel.Solver(cfg, tol=1e-8, max_it=20000)
        rho = torch.full((ne,), 0.4, dtype=torch.float64, device="cuda")
        ts = s.topopt_state(rho, volfrac=0.4, tol_eta=eta, tol_max=1e-3)
        hist, tols, its = [], [], 0
        for _ in range(steps):
            st = s.topopt_step(ts)
            hist.append(ts.compliance)
            tols.append(ts.tol_used)
            its += st.iters
        return hist, tols, its

    h_fix, t_fix, it_fix = run(0.0)
    h_ad, t_ad, it_ad = run(0.1)
    assert all(t == 1e-8 for t in t_fix)
    for k in range(len(h_ad)):
        assert t_ad[k] == topopt.adaptive_tolerance(h_ad[:k], 0.1, 1e-8, 1e-3), k
    assert min(t_ad) < 1e-3  # the tolerance tightens as the design settles
    assert abs(h_ad[-1] - h_fix[-1]) <= 5e-3 * h_fix[-1], (h_ad[-1], h_fix[-1])
    assert it_ad < 0.9 * it_fix, (it_ad, it_fix)


def test_history_guess_with_adaptive_tolerance():
    # the Galerkin guess of the last Picard solutions (HISTORY coarse space,
    # X0 only: no correction inside the iteration) with the adaptive
    # tolerance: the same rule on its own compliances, the fixed-tolerance
    # design's compliance, and fewer PCG iterations than the adaptive
    # tolerance started from zero
    from paper_1501_06211_gb300 import ddel
    cfg = _mbb(128, 64, 16)
    ne = int(np.prod(cfg["ne"]))

    def run(eta, learner_opts=None, steps=60):
        s = ddel.Solver(cfg, tol=1e-8, max_it=20000)
        L = ddel.Learner(s, **learner_opts) if learner_opts else None
        rho = torch.full((ne,), 0.4, dtype=torch.float64, device="cuda")
        ts = s.topopt_state(rho, volfrac=0.4, learner=L, tol_eta=eta, tol_max=1e-3)
        hist, tols, its = [], [], 0
        for _ in range(steps):
            st = s.topopt_step(ts)
            hist.append(ts.compliance)
            tols.append(ts.tol_used)
            its += st.iters
        if L is not None:
            L.close()
        s.close()
        return hist, tols, its

    h_fix, _, _ = run(0.0)
    _, _, it_ad = run(0.1)
    h_hx, t_hx, it_hx = run(0.1, dict(mode=ddel.DDEL_LEARN_HISTORY, k_history=4, coarse_flags=ddel.DDEL_COARSE_X0))
    for k in range(len(h_hx)):
        assert t_hx[k] == topopt.adaptive_tolerance(h_hx[:k], 0.1, 1e-8, 1e-3), k
    assert abs(h_hx[-1] - h_fix[-1]) <= 5e-3 * h_fix[-1], (h_hx[-1], h_fix[-1])
    assert it_hx < 0.8 * it_ad, (it_hx, it_ad)


def test_table3_sweep_trends():
    # Table 3's study on the built kernels (cantilever, OC, adaptive
    # tolerance, the variable-thickness sheet p = 1 of Sec. 5): Picard steps
    # to max |rho_new - rho| < 0.01 and average PCG iterations per step
    # against h and the number of subdomains (8, 32, 128: square subdomains
    # on the 2 x 1 beam, reading Q24).  At a fixed number of subdomains the
    # average PCG count stays nearly flat as h halves twice; it grows with the
    # number of subdomains.
    from paper_1501_06211_gb300 import ddel
    table = {}
    for nx in (32, 64, 128):
        for nsx in (4, 8, 16):
            sub = nx // nsx
            cfg = workloads.small_config(nx, nx // 2, sub, seed=None, p=1.0)
            ne = nx * nx // 2
            s = ddel.Solver(cfg, tol=1e-8, max_it=20000)
            rho = torch.full((ne,), 0.5, dtype=torch.float64, device="cuda")
            ts = s.topopt_state(rho, volfrac=0.5, tol_eta=0.1, tol_max=1e-3)
            its, steps = 0, 0
            while steps < 100:
                st = s.topopt_step(ts)
                its += st.iters
                steps += 1
                if ts.change < 0.01:
                    break
            table[(nx, nsx)] = (steps, its / steps)
            s.close()
    print("Table 3 sweep: (Picard steps, mean PCG iterations)")
    for nx in (32, 64, 128):
        print(f"h = 1/{nx // 2}: " + "  ".join(f"{table[(nx, n)][0]:3d} ({table[(nx, n)][1]:5.1f})"
                                              for n in (4, 8, 16)))
    for nsx in (4, 8, 16):
        a = [table[(nx, nsx)][1] for nx in (32, 64, 128)]
        assert a[2] <= 2.0 * a[0], (nsx, a)
    for nx in (32, 64, 128):
        b = [table[(nx, n)][1] for n in (4, 8, 16)]
        assert b[0] <= b[1] <= b[2], (nx, b)
