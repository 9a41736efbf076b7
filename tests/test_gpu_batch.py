"""Batched independent problems of uneven size (one stream per problem, or one
persistent launch with a device work queue).

Every problem of the batch is compared with the oracle's direct solve and
with its own ddel_solve, which it must reproduce bitwise (same kernels in the
same order, deterministic reductions)."""
import numpy as np
import pytest

import workloads
from oracle import direct, fem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problems():
    probs = [p for p in workloads.batch_problems(base_seed=0, count=64) if p["ne"][0] <= 128]
    return probs[:8]


@pytest.mark.parametrize("persistent", [False, True], ids=["streams", "persistent"])
def test_batch_matches_oracle_and_single_solves(persistent):
    # streams: one stream per problem; persistent: one persistent launch per
    # batch of iterations with the device work queue (the same blocks, the
    # same bits)
    from paper_1501_06211_gb300 import ddel
    probs = _problems()
    assert len(probs) >= 4 and len({p["sub"] for p in probs}) >= 2
    solvers, us, refs = [], [], []
    for cfg in probs:
        s = ddel.Solver(cfg, tol=1e-10, max_it=20000)
        rho = workloads.density(cfg)
        s.assemble(rho)
        solvers.append(s)
        us.append(torch.zeros(s.n_dof, dtype=torch.float64, device="cuda"))
        grid = fem.Grid(2, *cfg["ne"])
        fixed, f = fem.bc_from_spec(grid, cfg["bc"])
        K = fem.assemble(grid, fem.element_stiffness(2, 1.0, cfg["nu"]),
                         fem.element_factors(rho, cfg["E"], cfg["p"]))
        refs.append((direct.solve(K, f, fixed), K, f, fixed))
    code, sts = ddel.ddel_batch_solve([s.h for s in solvers], us, persistent=persistent)
    assert code == 0, [st.as_dict() for st in sts]
    for s, u, (u_ref, K, f, fixed), st in zip(solvers, us, refs, sts):
        un = u.cpu().numpy()
        assert st.relres <= 1e-10, st.as_dict()
        assert np.linalg.norm(un - u_ref) <= 1e-8 * np.linalg.norm(u_ref)
        # the single-problem path gives the same bits
        s.factor()
        u1 = torch.zeros_like(u)
        s.solve(None, u1)
        assert torch.equal(u1, u)


def test_autotune_choice_cache_and_parity(tmp_path):
    # the autotuner times the Schur forms on this GPU, applies the winner,
    # caches it; the tuned solve still matches the oracle
    from paper_1501_06211_gb300 import ddel
    cfg = workloads.small_config(128, 64, 16, seed=11)
    rho = workloads.density(cfg)
    s = ddel.Solver(cfg, tol=1e-10, max_it=20000)
    s.assemble(rho)
    cache = str(tmp_path / "tune.txt")
    code, mode, check, cached = ddel.ddel_autotune(s.h, cache)
    assert code == 0 and not cached
    assert mode in (0, 1, 2) and check in (8, 16, 32)
    lines = open(cache).read().strip().splitlines()
    assert len(lines) == 1
    # key (dim sub BP n_sub precision), then mode, check_every, tensor_form,
    # schur_split (CTAs per subdomain of the FP64 explicit apply)
    fields = lines[0].split()
    assert len(fields) == 9 and int(fields[5]) == mode and int(fields[6]) == check
    assert fields[7] in ("0", "1") and fields[8] in ("0", "1", "2", "4")
    s2 = ddel.Solver(cfg, tol=1e-10, max_it=20000)
    s2.assemble(rho)
    code2, mode2, check2, cached2 = ddel.ddel_autotune(s2.h, cache)
    assert code2 == 0 and cached2 and (mode2, check2) == (mode, check)
    s2.factor()
    u, st = s2.solve()
    grid = fem.Grid(2, *cfg["ne"])
    fixed, f = fem.bc_from_spec(grid, cfg["bc"])
    K = fem.assemble(grid, fem.element_stiffness(2, 1.0, cfg["nu"]),
                     fem.element_factors(rho, cfg["E"], cfg["p"]))
    u_ref = direct.solve(K, f, fixed)
    assert np.linalg.norm(u - u_ref) <= 1e-8 * np.linalg.norm(u_ref)
