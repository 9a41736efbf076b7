"""GPU parity of the paper's own interface preconditioner and Krylov method
(Sec. 3-4, Table 1): the global H~_theta = M (M^-1 L)^(1-theta) on the whole
interface applied by inverse Lanczos with the inner PCG on L, and flexible
GMRES on the full system with the block-triangular preconditioner.

Step by step against `oracle/globalprec.py` (inner="pcg"): the Lanczos
tridiagonal T_m, the inner iteration counts and z = S~^-1 r; whole solves
against `oracle/krylov.py: fgmres` (iteration counts) and the direct solve;
and Table 1's study on the built kernels: S~ = I, the face-local and the
global H~_0.5 and H~_OPT on the Q14 problem, counts equal to the oracle's.
"""
import numpy as np
import pytest

import workloads
from oracle import dd, direct, fem, globalprec, krylov

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


_SYSTEMS = {}


def get(cfg):
    """The oracle's system of a workload description (cached by its repr)."""
    k = repr(sorted(cfg.items()))
    if k not in _SYSTEMS:
        grid = fem.Grid(2, *cfg["ne"])
        fixed, f = fem.bc_from_spec(grid, cfg["bc"])
        Ke = fem.element_stiffness(2, 1.0, cfg["nu"])
        fac = fem.element_factors(workloads.density(cfg), cfg["E"], cfg["p"])
        dec, K, dds = dd.build(grid, cfg["sub"], fixed, Ke, fac)
        _SYSTEMS[k] = (cfg, grid, fixed, f, dec, K, dds)
    return _SYSTEMS[k]


def solver(cfg, theta=0.5):
    from paper_1501_06211_gb300 import ddel
    s = ddel.Solver(cfg, theta=theta)
    s.assemble(workloads.density(cfg))
    s.factor()
    return s


def perm_of(s, dec):
    gd = s.gamma_dofs()
    pos = {int(v): k for k, v in enumerate(dec.gamma_dofs)}
    return np.array([pos[int(v)] for v in gd])  # library order -> oracle order


def full_system(dec, K, dds, f):
    I = np.concatenate([b[0] for b in dds.blocks])
    order = np.concatenate([I, dec.gamma_dofs])
    return K[order][:, order], f[order]


CASES = {
    "cantilever_32x16_s8": workloads.small_config(32, 16, 8, p=1.0),
    "grf_64x32_s8": workloads.small_config(64, 32, 8, seed=2),
    "table1_h32_n8": workloads.table1_config(32, 4),
}


@pytest.mark.parametrize("scaling", [0, 1], ids=["paper_literal", "diag_surrogate"])
@pytest.mark.parametrize("name", list(CASES))
def test_global_precond_step_by_step(name, scaling):
    from paper_1501_06211_gb300 import ddel
    if name.startswith("grf") and scaling == 0:
        pytest.skip("heterogeneous material needs the scaling (reading Q25)")
    cfg, grid, fixed, f, dec, K, dds = get(CASES[name])
    s = solver(cfg)
    perm = perm_of(s, dec)
    r_lib = np.random.default_rng(3).standard_normal(s.n_gamma)
    r_or = np.zeros_like(r_lib)
    r_or[perm] = r_lib
    opt = ddel.ddel_default_gmres_options(lanczos_steps=8, inner_tol=1e-3, mass_tol=1e-14,
                                          global_scaling=scaling)
    z = torch.zeros(s.n_gamma, dtype=torch.float64, device="cuda")
    code, rec = ddel.ddel_global_precond_apply(s.h, opt, torch.as_tensor(r_lib, device="cuda"), z,
                                               with_record=True)
    assert code == 0
    def oracle(rv):
        gp = globalprec.GlobalPreconditioner(dec, K, 0.5, steps=8, face_scaling="diag" if scaling else False,
                                             inner="pcg", inner_tol=1e-3)
        return gp.apply(rv), gp.comps

    z_ref, comps = oracle(r_or)
    # the inexact inner solves (tolerance 1e-3) make the Lanczos recurrence
    # sensitive to rounding: the oracle's own change under a 1e-15 relative
    # perturbation of r sets the scale of the comparison (at least 1e-9)
    z_p, comps_p = oracle(r_or * (1 + 1e-15 * np.random.default_rng(5).standard_normal(len(r_or))))
    spread_z = np.linalg.norm(z_p - z_ref) / np.linalg.norm(z_ref)
    for c, comp in enumerate(comps):
        a_ref, b_ref = comp.last_T
        spread_a = np.max(np.abs(comps_p[c].last_T[0] - a_ref) / np.abs(a_ref))
        tol = max(1e-9, 20 * spread_a)
        assert rec[c]["m"] == len(a_ref)
        assert rec[c]["inner_its"] == comp.inner_its, (rec[c]["inner_its"], comp.inner_its)
        assert np.allclose(rec[c]["alpha"], a_ref, rtol=tol, atol=0), (tol, rec[c]["alpha"], a_ref)
        assert np.allclose(rec[c]["beta"], b_ref, rtol=10 * tol, atol=1e-12 * np.abs(a_ref).max())
        if not name.startswith("grf"):  # 4 x 2 subdomains, as the paper's smallest cases
            # the paper's inner iteration range (Sec. 4: "typically between 2 and 12")
            assert max(comp.inner_its) <= 12
    zl = z.cpu().numpy()
    assert np.linalg.norm(zl - z_ref[perm]) <= max(1e-9, 20 * spread_z) * np.linalg.norm(z_ref), spread_z


@pytest.mark.parametrize("precond", ["identity", "face", "global"])
@pytest.mark.parametrize("s_edge", [4, 8])
def test_fgmres_counts_and_solution_match_oracle(precond, s_edge):
    # the oracle's Table-1 set-up of test_oracle_globalprec: 4 x 2 subdomains,
    # full-system FGMRES to 1e-6 with the block-triangular preconditioner
    from paper_1501_06211_gb300 import ddel
    cfg = workloads.small_config(4 * s_edge, 2 * s_edge, s_edge, p=1.0)
    cfg, grid, fixed, f, dec, K, dds = get(cfg)
    Kp, b = full_system(dec, K, dds, f)
    if precond == "identity":
        apply = lambda v: v  # noqa: E731
    elif precond == "face":
        apply = dd.FacePreconditioner(dec, K, 0.5).apply
    else:
        apply = globalprec.GlobalPreconditioner(dec, K, 0.5, steps=8, face_scaling="diag", inner="pcg",
                                                inner_tol=1e-3).apply
    _, k_ref, _ = krylov.fgmres(lambda v: Kp @ v, krylov.block_right_preconditioner(dds, apply), b, 1e-6, 300)
    s = solver(cfg)
    code = {"identity": ddel.DDEL_PREC_IDENTITY, "face": ddel.DDEL_PREC_FACE, "global": ddel.DDEL_PREC_GLOBAL}
    u, st = s.gmres(precond=code[precond], lanczos_steps=8, inner_tol=1e-3, mass_tol=1e-14, tol=1e-6,
                    max_it=300)
    assert st.status == 0, st.as_dict()
    assert abs(st.iters - k_ref) <= 1, (st.iters, k_ref)
    assert st.relres <= 2e-6, st.as_dict()
    u_ref = direct.solve(K, f, fixed)
    assert np.linalg.norm(u - u_ref) <= 1e-4 * np.linalg.norm(u_ref)
    # tighter: the same Krylov method converges to the direct solution
    u2, st2 = s.gmres(precond=code[precond], lanczos_steps=8, inner_tol=1e-3, mass_tol=1e-14, tol=1e-11,
                      max_it=300)
    assert np.linalg.norm(u2 - u_ref) <= 1e-8 * np.linalg.norm(u_ref), st2.as_dict()


def test_table1_study_on_the_q14_problem():
    # Table 1 (Sec. 4) on the built kernels, on the problem of reading Q14:
    # iterations of full-system FGMRES (tol 1e-6) with S~ = I grow as h
    # shrinks; with the global H~_theta (inverse Lanczos, 8 steps, inner PCG
    # 1e-3) they grow much more slowly and are far fewer; the global form's
    # count equals the oracle's FGMRES with the same preconditioner (+-1).
    # H~_OPT (theta 0.6 for 32 subdomains) is run and reported, not asserted
    # better: on this reading of the problem it takes more iterations
    from paper_1501_06211_gb300 import ddel
    rows = {}
    for n_x, theta_opt in ((4, 0.5), (8, 0.6)):
        for h_inv in (16, 32, 64):
            cfg = workloads.table1_config(h_inv, n_x)
            if cfg["sub"] < 2:
                continue
            cfg, grid, fixed, f, dec, K, dds = get(cfg)
            row = {}
            for name, pc, theta in (("I", ddel.DDEL_PREC_IDENTITY, 0.5), ("H0.5", ddel.DDEL_PREC_GLOBAL, 0.5),
                                    ("HOPT", ddel.DDEL_PREC_GLOBAL, theta_opt)):
                s = solver(cfg, theta=theta)
                _, st = s.gmres(precond=pc, lanczos_steps=8, inner_tol=1e-3, mass_tol=1e-14, tol=1e-6,
                                global_scaling=0, max_it=400)
                assert st.status == 0, (h_inv, n_x, name, st.as_dict())
                row[name] = st.iters
                s.close()
            if h_inv <= 32:  # the oracle's count for the global form (dense eigensolves: small grids)
                Kp, b = full_system(dec, K, dds, f)
                gp = globalprec.GlobalPreconditioner(dec, K, 0.5, steps=8, face_scaling=False, inner="pcg",
                                                     inner_tol=1e-3)
                k_ref = krylov.fgmres(lambda v: Kp @ v, krylov.block_right_preconditioner(dds, gp.apply), b,
                                      1e-6, 400)[1]
                assert abs(row["H0.5"] - k_ref) <= 1, (h_inv, n_x, row, k_ref)
            rows[(n_x, h_inv)] = row
    for n_x in (4, 8):
        its = [rows[(n_x, h)] for h in (16, 32, 64) if (n_x, h) in rows]
        grow_i = its[-1]["I"] / its[0]["I"]
        grow_h = its[-1]["H0.5"] / its[0]["H0.5"]
        assert grow_i > 1.25 and grow_h < grow_i / 1.3, its
        assert its[-1]["H0.5"] < its[-1]["I"] / 1.5, its
        assert all(r["HOPT"] > 0 for r in its), its


def test_singular_interface_laplacian_is_rejected():
    # one row of subdomains: the interface lines miss the clamped edge, so L
    # is singular (reading Q5's case) and the GPU form refuses it
    from paper_1501_06211_gb300 import ddel
    cfg = workloads.small_config(64, 16, 16, seed=4)
    s = solver(cfg)
    _, st = None, None
    opt = ddel.ddel_default_gmres_options()
    z = torch.zeros(s.n_gamma, dtype=torch.float64, device="cuda")
    r = torch.ones_like(z)
    code, _ = ddel.ddel_global_precond_apply(s.h, opt, r, z)
    assert code == ddel.DDEL_EINVAL
