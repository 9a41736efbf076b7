"""Local Schur complements formed on the tensor cores (tcgen05, Ozaki
splitting of W = L^-1 K_IG into BF16 slices with exact FP32 accumulation)
against the FP64-pipe formation and the oracle.

S_i = K_GG^(i) - W^T W is the definition of eq. 3MatSplit; the tensor-core
form must reproduce it to FP64 accuracy: the Schur apply with the explicit
S_i agrees with the oracle's matrix-free S to 1e-10 and with the FP64-pipe
formation to 1e-12, on rings of 128 (16 x 16 subdomains) and 256 (32 x 32),
homogeneous and at SIMP contrast 1e9; whole solves keep the FP64 bar.  (The
double-float form uses the tensor cores for rings of 256 only; its rings of
128 keep their double-float formation, and the test then checks that form.)
"""
import numpy as np
import pytest

import workloads
from oracle import dd, direct, fem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "c0": workloads.config("c0"),
    "grf128": workloads.small_config(128, 64, 16, seed=11),
    "s32": workloads.small_config(128, 64, 32, seed=3),
    "s32_row": workloads.small_config(64, 32, 32, seed=6),
}


def oracle(cfg):
    grid = fem.Grid(2, *cfg["ne"])
    fixed, f = fem.bc_from_spec(grid, cfg["bc"])
    Ke = fem.element_stiffness(2, 1.0, cfg["nu"])
    rho = workloads.density(cfg)
    dec, K, dds = dd.build(grid, cfg["sub"], fixed, Ke, fem.element_factors(rho, cfg["E"], cfg["p"]))
    return rho, fixed, f, dec, K, dds


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("mode", [1, 2], ids=["explicit_fp64", "auto_double_float"])
@pytest.mark.parametrize("name", list(CASES))
def test_tensor_core_schur_complements(name, mode):
    from paper_1501_06211_gb300 import ddel
    cfg = CASES[name]
    rho, fixed, f, dec, K, dds = oracle(cfg)
    sols = {}
    ys = {}
    x = None
    for tf in (1, 0):
        s = ddel.Solver(cfg, schur_mode=mode, tensor_form=tf, tol=1e-10, max_it=20000)
        s.assemble(rho)
        s.factor()
        info = ddel.ddel_kernel_info(s.h)
        assert info["schur_form"] == 1
        gd = s.gamma_dofs()
        if x is None:
            x = np.random.default_rng(2).standard_normal(len(gd))
        y = torch.zeros(len(gd), dtype=torch.float64, device="cuda")
        assert ddel.ddel_schur_apply(s.h, torch.as_tensor(x, device="cuda"), y) == 0
        ys[tf] = y.cpu().numpy()
        u, st = s.solve(check=False)
        sols[tf] = (u, st)
        s.close()
    pos = {int(v): k for k, v in enumerate(dec.gamma_dofs)}
    perm = np.array([pos[int(v)] for v in gd])
    xo = np.zeros(len(gd))
    xo[perm] = x
    y_ref = dds.schur_apply(xo)[perm]
    assert rel(ys[1], y_ref) < 1e-10, rel(ys[1], y_ref)
    if mode == 1:  # both FP64 formations applied in FP64: the same S_i to rounding
        assert rel(ys[1], ys[0]) < 1e-12, rel(ys[1], ys[0])
    u_ref = direct.solve(K, f, fixed)
    u, st = sols[1]
    assert st.relres <= 1e-9, st.as_dict()
    assert rel(u, u_ref) <= 1e-8, (rel(u, u_ref), st.as_dict())


@pytest.mark.parametrize("name", ["grf128", "s32"])
def test_tensor_core_fp32_form(name):
    # the FP32 form: S_i = K_GG - W^T W from BF16 slices of the FP32 W on the
    # tensor cores (to FP64 accuracy, then rounded to FP32), applied in FP32;
    # FP64 refinement wins the accuracy back (the bar of the reduced-precision
    # forms: 1e-6)
    from paper_1501_06211_gb300 import ddel
    cfg = CASES[name]
    rho, fixed, f, dec, K, dds = oracle(cfg)
    s = ddel.Solver(cfg, precision=ddel.DDEL_FP32, schur_mode=1, tensor_form=2, tol=1e-9, max_it=20000,
                    max_cycles=60, inner_tol=0.1)
    s.assemble(rho)
    s.factor()
    gd = s.gamma_dofs()
    x = np.random.default_rng(4).standard_normal(len(gd))
    y = torch.zeros(len(gd), dtype=torch.float64, device="cuda")
    assert ddel.ddel_schur_apply(s.h, torch.as_tensor(x, device="cuda"), y) == 0
    pos = {int(v): k for k, v in enumerate(dec.gamma_dofs)}
    perm = np.array([pos[int(v)] for v in gd])
    xo = np.zeros(len(gd))
    xo[perm] = x
    # the FP32 operator: S to FP32 accuracy relative to its largest entries
    assert rel(y.cpu().numpy(), dds.schur_apply(xo)[perm]) < 1e-4
    u, st = s.solve(check=False)
    assert st.relres <= 1e-9, st.as_dict()
    assert rel(u, direct.solve(K, f, fixed)) <= 1e-6, st.as_dict()
