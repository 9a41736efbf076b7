"""GPU parity of the 3D H8 path against the oracle.

Small grids (several subdomains, boundary planes of different sizes, padded
blocks; one of them with the 8^3-element subdomains of the 96x48x48 workload)
are compared element by element at every step and for the full solve;
the full 96x48x48 workload (432 subdomains of 8^3) is checked through the
residual computed by the oracle's own matrix-free K(rho).
"""
import functools

import numpy as np
import pytest

import workloads
from oracle import dd, direct, fem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "3d_16x8x8_s4": workloads.small_config(16, 8, 4, seed=1, nz=8),
    "3d_12x12x8_s4": workloads.small_config(12, 12, 4, seed=2, nz=8),
    # the subdomains of the 96x48x48 workload (8^3 elements): the middle ones
    # have interior planes of 7 x 7 nodes (147 DOFs), as there
    "3d_16x24x24_s8": workloads.small_config(16, 24, 8, seed=3, nz=24),
}


@functools.lru_cache(maxsize=None)
def oracle_system(name):
    cfg = CASES[name]
    grid = fem.Grid(3, *cfg["ne"])
    fixed, f = fem.bc_from_spec(grid, cfg["bc"])
    Ke = fem.element_stiffness(3, 1.0, cfg["nu"])
    rho = workloads.density(cfg)
    fac = fem.element_factors(rho, cfg["E"], cfg["p"])
    dec, K, dds = dd.build(grid, cfg["sub"], fixed, Ke, fac)
    pre = dd.FacePreconditioner(dec, K)
    u_ref = direct.solve(K, f, fixed)
    return dict(cfg=cfg, grid=grid, fixed=fixed, f=f, rho=rho, dec=dec, K=K, dds=dds, pre=pre,
                u_ref=u_ref)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def solver(name, **opts):
    from paper_1501_06211_gb300 import ddel
    o = oracle_system(name)
    s = ddel.Solver(o["cfg"], **opts)
    s.assemble(o["rho"])
    s.factor()
    return s, o


@pytest.mark.parametrize("name", list(CASES))
def test_3d_steps(name):
    from paper_1501_06211_gb300 import ddel
    s, o = solver(name)
    gd = s.gamma_dofs()
    og = o["dec"].gamma_dofs
    assert sorted(gd.tolist()) == og.tolist()
    pos = {int(v): k for k, v in enumerate(og)}
    perm = np.array([pos[int(v)] for v in gd])
    n = o["grid"].n_dof
    x = np.random.default_rng(0).standard_normal(n)
    x[o["fixed"]] = 0
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    assert ddel.ddel_apply_K(s.h, dev(x), y) == 0
    ref = o["K"] @ x
    ref[o["fixed"]] = 0
    assert rel(y.cpu().numpy(), ref) < 1e-13
    g = torch.zeros(len(gd), dtype=torch.float64, device="cuda")
    assert ddel.ddel_condense(s.h, dev(o["f"]), g) == 0
    assert rel(g.cpu().numpy(), o["dds"].condense(o["f"])[perm]) < 1e-10
    xg = np.random.default_rng(1).standard_normal(len(gd))
    xo = np.zeros(len(og))
    xo[perm] = xg
    yg = torch.zeros_like(g)
    assert ddel.ddel_schur_apply(s.h, dev(xg), yg) == 0
    assert rel(yg.cpu().numpy(), o["dds"].schur_apply(xo)[perm]) < 1e-10
    z = torch.zeros_like(g)
    assert ddel.ddel_precond_apply(s.h, dev(xg), z) == 0
    assert rel(z.cpu().numpy(), o["pre"].apply(xo)[perm]) < 1e-12
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    assert ddel.ddel_back_substitute(s.h, dev(o["f"]), dev(xg), u) == 0
    assert rel(u.cpu().numpy(), o["dds"].back_substitute(o["f"], xo)) < 1e-10


@pytest.mark.parametrize("theta", [0.5, 0.3], ids=["theta_half", "theta_hopt"])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
def test_3d_solve(name, prec, theta):
    s, o = solver(name, precision=prec, tol=1e-10, max_it=20000, theta=theta)
    u, st = s.solve(check=False)
    assert st.relres <= 1e-9, st.as_dict()
    assert rel(u, o["u_ref"]) <= (1e-8 if prec == 0 else 1e-6), st.as_dict()


@pytest.mark.parametrize("name", list(CASES))
def test_3d_tensor_core_factor_planes(name):
    # C_k C_k^T of every plane on the tensor cores (tensor_form = 2: Ozaki
    # slices of C_k, FP64 accuracy): the Schur complement and the solve keep
    # the bars of the FP64-pipe factorisation
    from paper_1501_06211_gb300 import ddel
    s, o = solver(name, tensor_form=2, tol=1e-10, max_it=20000)
    gd = s.gamma_dofs()
    pos = {int(v): k for k, v in enumerate(o["dec"].gamma_dofs)}
    perm = np.array([pos[int(v)] for v in gd])
    xg = np.random.default_rng(1).standard_normal(len(gd))
    xo = np.zeros(len(gd))
    xo[perm] = xg
    yg = torch.zeros(len(gd), dtype=torch.float64, device="cuda")
    assert ddel.ddel_schur_apply(s.h, dev(xg), yg) == 0
    assert rel(yg.cpu().numpy(), o["dds"].schur_apply(xo)[perm]) < 1e-10
    u, st = s.solve(check=False)
    assert st.relres <= 1e-9, st.as_dict()
    assert rel(u, o["u_ref"]) <= 1e-8, st.as_dict()


def test_3d_full_size_config2_residual():
    # 96 x 48 x 48 H8, 432 subdomains of 8^3, uniform-random densities: the
    # oracle's matrix-free K checks the residual of the GPU solution
    from paper_1501_06211_gb300 import ddel
    cfg = workloads.config("c2")
    grid = fem.Grid(3, *cfg["ne"])
    fixed, f = fem.bc_from_spec(grid, cfg["bc"])
    rho = workloads.density(cfg)
    Ke = fem.element_stiffness(3, 1.0, cfg["nu"])
    fac = fem.element_factors(rho, 1.0, cfg["p"])
    s = ddel.Solver(cfg, tol=1e-8, max_it=40000)
    s.assemble(rho)
    s.factor()
    u, st = s.solve(check=False)
    r = f - fem.apply_ebe(grid, Ke, fac, np.where(fixed, 0.0, u))
    r[fixed] = 0.0
    rr = np.linalg.norm(r) / np.linalg.norm(f)
    assert rr <= 1e-8, (rr, st.as_dict())
