"""GPU parity: every step of the CUDA path against the oracle, element by element.

All calls go through the C ABI (ctypes binding); the oracle runs on the CPU on
the same seeded inputs.  Tolerances: FP64 steps to 1e-10 relative (rounding
order differs), full FP64 solves to a relative displacement error <= 1e-8,
reduced-precision solves (FP32 factors + FP64 refinement) to <= 1e-6.
"""
import functools

import numpy as np
import pytest

import workloads
from oracle import dd, direct, fem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "c0": workloads.config("c0"),
    "grf128": workloads.small_config(128, 64, 16, seed=11),
    "mbb64_s8": workloads.small_config(64, 32, 8, seed=5, bc="mbb"),
    "s32": workloads.small_config(128, 64, 32, seed=3),
    # one row of 32 x 32 subdomains: 33 interior rows per plane (blocks of 96)
    "s32_row": workloads.small_config(64, 32, 32, seed=6),
    "onerow": workloads.small_config(64, 16, 16, seed=4),
}


@functools.lru_cache(maxsize=None)
def oracle_system(name):
    cfg = CASES[name]
    grid = fem.Grid(cfg["dim"], *cfg["ne"])
    fixed, f = fem.bc_from_spec(grid, cfg["bc"])
    Ke = fem.element_stiffness(cfg["dim"], 1.0, cfg["nu"])
    rho = workloads.density(cfg)
    fac = fem.element_factors(rho, cfg["E"], cfg["p"])
    dec, K, dds = dd.build(grid, cfg["sub"], fixed, Ke, fac)
    pre = dd.FacePreconditioner(dec, K)
    u_ref = direct.solve(K, f, fixed)
    return dict(cfg=cfg, grid=grid, fixed=fixed, f=f, rho=rho, dec=dec, K=K, dds=dds, pre=pre,
                u_ref=u_ref)


def solver(name, **opts):
    from paper_1501_06211_gb300 import ddel
    o = oracle_system(name)
    s = ddel.Solver(o["cfg"], **opts)
    s.assemble(o["rho"])
    s.factor()
    return s, o


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def to_global(vals, gdofs, n):
    out = np.zeros(n)
    out[gdofs] = vals
    return out


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("name", ["c0", "grf128", "mbb64_s8"])
def test_apply_K(name):
    from paper_1501_06211_gb300 import ddel
    s, o = solver(name)
    x = np.random.default_rng(0).standard_normal(o["grid"].n_dof)
    x[o["fixed"]] = 0
    y = torch.zeros(o["grid"].n_dof, dtype=torch.float64, device="cuda")
    assert ddel.ddel_apply_K(s.h, dev(x), y) == 0
    torch.cuda.synchronize()
    ref = o["K"] @ x
    ref[o["fixed"]] = 0
    assert rel(y.cpu().numpy(), ref) < 1e-13


@pytest.mark.parametrize("mode", [0, 1, 2], ids=["implicit", "explicit", "auto_double_float"])
@pytest.mark.parametrize("name", list(CASES))
def test_condense_schur_precond_backsub(name, mode):
    from paper_1501_06211_gb300 import ddel
    s, o = solver(name, schur_mode=mode)
    gd = s.gamma_dofs()
    og = o["dec"].gamma_dofs
    n = o["grid"].n_dof
    assert sorted(gd.tolist()) == og.tolist()
    pos = {int(v): k for k, v in enumerate(og)}
    perm = np.array([pos[int(v)] for v in gd])  # library order -> oracle order
    # condensed right-hand side (eq. 3MatSplit2, second line)
    g = torch.zeros(len(gd), dtype=torch.float64, device="cuda")
    assert ddel.ddel_condense(s.h, dev(o["f"]), g) == 0
    g_ref = o["dds"].condense(o["f"])
    assert rel(g.cpu().numpy(), g_ref[perm]) < 1e-10
    # Schur complement applied without forming it
    rng = np.random.default_rng(1)
    xg = rng.standard_normal(len(gd))
    y = torch.zeros_like(g)
    assert ddel.ddel_schur_apply(s.h, dev(xg), y) == 0
    xo = np.zeros(len(og))
    xo[perm] = xg
    assert rel(y.cpu().numpy(), o["dds"].schur_apply(xo)[perm]) < 1e-10
    # face-local preconditioner
    z = torch.zeros_like(g)
    assert ddel.ddel_precond_apply(s.h, dev(xg), z) == 0
    assert rel(z.cpu().numpy(), o["pre"].apply(xo)[perm]) < 1e-12
    # back substitution
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    assert ddel.ddel_back_substitute(s.h, dev(o["f"]), dev(xg), u) == 0
    u_ref = o["dds"].back_substitute(o["f"], xo)
    assert rel(u.cpu().numpy(), u_ref) < 1e-10


@pytest.mark.parametrize("mode", [0, 2], ids=["implicit", "auto"])
@pytest.mark.parametrize("name", list(CASES))
def test_solve_fp64_matches_direct(name, mode):
    # 1e-10: with SIMP contrast 1e9 (and the weakly supported MBB beam) the
    # FP64 residual floor lies between 2e-12 and 5e-10
    s, o = solver(name, tol=1e-10, schur_mode=mode, max_it=20000)
    u, st = s.solve(check=False)
    err = rel(u, o["u_ref"])
    assert st.relres <= 1e-9, st.as_dict()
    e = u - o["u_ref"]
    err_energy = np.sqrt(max(e @ (o["K"] @ e), 0.0) / (o["u_ref"] @ (o["K"] @ o["u_ref"])))
    assert err_energy <= 1e-8, (err_energy, st.as_dict())
    # displacement error: 1e-8, except on the weakly supported MBB beam with
    # contrast 1e9, where the residual floor (5e-10) times its conditioning
    # puts both solvers' own errors near 1e-8 (reading Q13: energy norm above)
    assert err <= (3e-8 if name.startswith("mbb") else 1e-8), (err, st.as_dict())
    # the residual computed by the oracle's own sparse K agrees
    assert direct.rel_residual(o["K"], o["f"], u, o["fixed"]) <= 1e-9


@pytest.mark.parametrize("mode", [0, 2], ids=["implicit", "auto"])
@pytest.mark.parametrize("name", ["c0", "grf128", "mbb64_s8", "s32"])
def test_solve_fp32_refined(name, mode):
    from paper_1501_06211_gb300 import ddel
    s, o = solver(name, precision=ddel.DDEL_FP32, tol=1e-9, schur_mode=mode, max_it=20000)
    u, st = s.solve(check=False)
    assert st.relres <= 1e-9, st.as_dict()
    assert rel(u, o["u_ref"]) <= 1e-6, st.as_dict()


def test_iterations_match_oracle_pcg():
    # Same algorithm, same stopping test: ||r_G|| <= 0.5 tol ||f||.
    s, o = solver("c0", tol=1e-8)
    u, st = s.solve()
    _, it, _ = dd.dd_solve(o["dds"], o["pre"], o["f"], tol=0.5e-8, ref="f")
    assert st.cycles == 1
    assert abs(st.iters - it) <= 1, (st.iters, it)


def test_device_and_host_paths_agree_and_repeat():
    s, o = solver("grf128", tol=1e-10)
    u_host, _ = s.solve()
    u_dev = torch.zeros(o["grid"].n_dof, dtype=torch.float64, device="cuda")
    s.solve(dev(o["f"]), u_dev)
    u2 = torch.zeros_like(u_dev)
    s.solve(dev(o["f"]), u2)
    assert np.array_equal(u_dev.cpu().numpy(), u_host)
    assert torch.equal(u_dev, u2)  # deterministic reductions: bitwise repeatable


def test_error_paths():
    from paper_1501_06211_gb300 import ddel
    o = oracle_system("c0")
    s = ddel.Solver(o["cfg"])
    with pytest.raises(ddel.DDELError) as e:
        s.solve()
    assert e.value.code == ddel.DDEL_ESTATE
    bad = o["rho"].copy()
    bad[3] = -1.0
    with pytest.raises(ddel.DDELError) as e:
        s.assemble(bad)
    assert e.value.code == ddel.DDEL_EINVAL
    # device-side detection of a bad density
    s.assemble(dev(bad))
    with pytest.raises(ddel.DDELError) as e:
        s.factor()
    assert e.value.code == ddel.DDEL_EINVAL
    # iteration cap
    s2 = ddel.Solver(o["cfg"], max_it=3, max_cycles=1, check_every=1)
    s2.assemble(o["rho"])
    s2.factor()
    u, st = s2.solve(check=False)
    assert st.status == ddel.DDEL_ENOCONV


@functools.lru_cache(maxsize=None)
def config1_oracle():
    # 512x256 Q1, 512 subdomains, GRF densities: the oracle's sparse K(rho) and
    # its direct solution (SuperLU + 3 refinement steps with an
    # extended-precision residual)
    cfg = workloads.config("c1")
    grid = fem.Grid(2, *cfg["ne"])
    fixed, f = fem.bc_from_spec(grid, cfg["bc"])
    rho = workloads.density(cfg)
    Ke = fem.element_stiffness(2, 1.0, cfg["nu"])
    K = fem.assemble(grid, Ke, fem.element_factors(rho, 1.0, 3.0))
    u_ref = direct.solve(K, f, fixed, refine=3)
    return cfg, rho, K, f, fixed, u_ref


@pytest.mark.parametrize("theta", [0.5, 0.6], ids=["theta_half", "theta_hopt"])
@pytest.mark.parametrize("prec,mode", [(0, 1), (0, 2), (1, 2)],
                         ids=["fp64_native", "fp64_double_float", "fp32_refined"])
def test_full_size_config1_parity(prec, mode, theta):
    # The full 512x256 workload solved tighter than the benchmark's 1e-8
    # (reading Q13: forward error can exceed the residual at contrast 1e9),
    # then held to the stated bars against the oracle's direct solution:
    # displacement and energy-norm error <= 1e-8 for the FP64 operator (native
    # or double-float), <= 1e-6 after refinement for the FP32 form.
    from paper_1501_06211_gb300 import ddel
    cfg, rho, K, f, fixed, u_ref = config1_oracle()
    assert direct.rel_residual(K, f, u_ref, fixed) <= 1e-10  # the FP64 evaluation floor: ~1e-11
    s = ddel.Solver(cfg, precision=prec, schur_mode=mode, tol=1e-10, max_it=20000, max_cycles=60,
                    inner_tol=0.1, theta=theta)
    s.assemble(rho)
    s.factor()
    u, st = s.solve(check=False)
    rr = direct.rel_residual(K, f, u, fixed)
    assert rr <= 1e-9, (rr, st.as_dict())
    e = u - u_ref
    err = rel(u, u_ref)
    err_energy = np.sqrt(max(e @ (K @ e), 0.0) / (u_ref @ (K @ u_ref)))
    bar = 1e-8 if prec == 0 else 1e-6
    assert err <= bar and err_energy <= bar, (err, err_energy, st.as_dict())


def test_full_size_config1_sampled_at_bench_tolerance():
    # the benchmark's own launch configuration (tol 1e-8, native FP64 form,
    # theta = 0.6): the
    # residual under the oracle's K and sampled displacement entries
    from paper_1501_06211_gb300 import ddel
    cfg, rho, K, f, fixed, u_ref = config1_oracle()
    s = ddel.Solver(cfg, schur_mode=1, tol=1e-8, max_it=20000, inner_tol=0.1, max_cycles=60, theta=0.6)
    s.assemble(rho)
    s.factor()
    u, st = s.solve()
    assert st.status == 0
    assert direct.rel_residual(K, f, u, fixed) <= 1e-8
    idx = np.random.default_rng(7).choice(len(u), 2000, replace=False)
    scale = np.abs(u_ref).max()
    assert np.abs(u[idx] - u_ref[idx]).max() <= 1e-5 * scale


def test_schur_apply_ring_alone():
    # the Schur kernel alone (timing entry point): status codes, and the full
    # apply around it is unchanged bit for bit
    from paper_1501_06211_gb300 import ddel
    o = oracle_system("c0")
    s0 = ddel.Solver(o["cfg"])
    s0.assemble(o["rho"])
    x = torch.randn(s0.n_gamma, dtype=torch.float64, device="cuda")
    assert ddel.ddel_schur_apply_ring(s0.h, x) == ddel.DDEL_ESTATE  # before factor
    s0.factor()
    y1 = torch.zeros_like(x)
    y2 = torch.zeros_like(x)
    assert ddel.ddel_schur_apply(s0.h, x, y1) == 0
    assert ddel.ddel_schur_apply_ring(s0.h, x) == 0
    assert ddel.ddel_schur_apply(s0.h, x, y2) == 0
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
