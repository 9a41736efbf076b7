"""Pins of the oracle's coarse space (Galerkin x0 and additive correction)
against least squares, spectra and special cases that fix the answer."""
import numpy as np
import pytest

import workloads
from oracle import coarse, dd, fem


def spd(n, seed, cond=1e3):
    rng = np.random.default_rng(seed)
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.logspace(0, np.log10(cond), n)
    return (Qm * lam) @ Qm.T


def test_basis_drops_dependent_columns():
    rng = np.random.default_rng(0)
    a, b = rng.standard_normal(20), rng.standard_normal(20)
    Q = coarse.orthonormal_basis(np.stack([a, 2 * a, b, a - 3 * b], axis=1))
    assert Q.shape == (20, 2)
    assert np.allclose(Q.T @ Q, np.eye(2), atol=1e-14)


def test_galerkin_x0_is_energy_norm_best_approximation():
    # x0 minimises ||x* - x||_S over span(Z): least squares on L^T (S = L L^T)
    S = spd(30, 1)
    rng = np.random.default_rng(2)
    g = rng.standard_normal(30)
    Z = rng.standard_normal((30, 4))
    cs = coarse.CoarseSpace(lambda v: S @ v, Z)
    xs = np.linalg.solve(S, g)
    L = np.linalg.cholesky(S)
    c, *_ = np.linalg.lstsq(L.T @ Z, L.T @ xs, rcond=None)
    # the residual test may discard x0; compare the projection itself
    x0 = cs.Q @ cs.solve_E(cs.Q.T @ g)
    assert np.allclose(x0, Z @ c, rtol=1e-10, atol=1e-12)


def test_exact_solution_in_span_converges_in_zero_iterations():
    S = spd(25, 3)
    rng = np.random.default_rng(4)
    g = rng.standard_normal(25)
    xs = np.linalg.solve(S, g)
    Z = np.stack([rng.standard_normal(25), xs, rng.standard_normal(25)], axis=1)
    x, it, hist, cs = coarse.coarse_pcg(lambda v: S @ v, lambda r: r, g, Z, 1e-10, 100)
    assert it == 0
    assert np.allclose(x, xs, rtol=1e-10)


def test_additive_correction_shifts_the_deflated_eigenvalues_by_one():
    # P = I, Z = k eigenvectors of S: P_c S = S + Q Q^T has eigenvalues
    # lambda_i + 1 on span(Z) and lambda elsewhere
    n, k = 16, 3
    S = spd(n, 5, cond=50)
    lam, V = np.linalg.eigh(S)
    cs = coarse.CoarseSpace(lambda v: S @ v, V[:, :k])
    Pc = cs.preconditioner(lambda r: r)
    M = np.stack([Pc(S[:, j]) for j in range(n)], axis=1)
    ev = np.sort(np.linalg.eigvals(M).real)
    expect = np.sort(np.concatenate([lam[:k] + 1.0, lam[k:]]))
    assert np.allclose(ev, expect, rtol=1e-10)


def test_deflation_moves_the_deflated_eigenvalues_to_one():
    # P = I, Z = k eigenvectors of S: P_d S has eigenvalue 1 on span(Z) and
    # keeps lambda on the S-invariant complement
    n, k = 16, 3
    S = spd(n, 6, cond=50)
    lam, V = np.linalg.eigh(S)
    cs = coarse.CoarseSpace(lambda v: S @ v, V[:, :k])
    Pd = cs.deflated_preconditioner(lambda r: r)
    M = np.stack([Pd(S[:, j]) for j in range(n)], axis=1)
    ev = np.sort(np.linalg.eigvals(M).real)
    expect = np.sort(np.concatenate([np.ones(k), lam[k:]]))
    assert np.allclose(ev, expect, rtol=1e-10)


def test_indefinite_coarse_matrix_falls_back_to_plain_pcg():
    A = np.diag([1.0, -1.0, 2.0])
    cs = coarse.CoarseSpace(lambda v: A @ v, np.eye(3)[:, :2])
    assert not cs.spd
    assert cs.x0(np.ones(3)) is None
    r = np.array([1.0, 2.0, 3.0])
    assert np.array_equal(cs.preconditioner(lambda v: 2 * v)(r), 2 * r)


def test_x0_discarded_when_it_raises_the_residual():
    # S = diag(1, 100), Z = (1, 1), g = (1, 0): x0 = (1, 1) / 101 gives
    # ||g - S x0|| = sqrt((100/101)^2 + (100/101)^2) > 1 = ||g||
    S = np.diag([1.0, 100.0])
    cs = coarse.CoarseSpace(lambda v: S @ v, np.array([[1.0], [1.0]]))
    assert cs.x0(np.array([1.0, 0.0])) is None
    # g = (0, 1): ||r0|| = sqrt(2) / 101 < 1, kept
    x0 = cs.x0(np.array([0.0, 1.0]))
    assert np.allclose(x0, np.array([1.0, 1.0]) / 101.0)


@pytest.fixture(scope="module")
def small_dd():
    cfg = workloads.small_config(32, 16, 8, seed=7)
    grid = fem.Grid(2, *cfg["ne"])
    fixed, f = fem.bc_from_spec(grid, cfg["bc"])
    Ke = fem.element_stiffness(2, 1.0, cfg["nu"])
    rho = workloads.density(cfg)
    dec, K, dds = dd.build(grid, cfg["sub"], fixed, Ke, fem.element_factors(rho, cfg["E"], cfg["p"]))
    pre = dd.FacePreconditioner(dec, K)
    return dict(cfg=cfg, grid=grid, fixed=fixed, f=f, Ke=Ke, rho=rho, dec=dec, K=K, dds=dds, pre=pre)


def test_coarse_pcg_same_solution_and_fewer_iterations_with_history(small_dd):
    o = small_dd
    dds, pre = o["dds"], o["pre"]
    g = dds.condense(o["f"])
    tol = 1e-10
    x_ref, it_ref, _ = dd.pcg(dds.schur_apply, pre.apply, g, tol, 5000)
    # coarse space from the solutions of perturbed densities (a Picard history)
    rng = np.random.default_rng(9)
    Zs = []
    for j in range(3):
        rho_j = np.clip(o["rho"] * np.exp(0.05 * rng.standard_normal(o["rho"].shape)), 1e-3, 1)
        _, _, dds_j = dd.build(o["grid"], o["cfg"]["sub"], o["fixed"], o["Ke"],
                               fem.element_factors(rho_j, o["cfg"]["E"], o["cfg"]["p"]))
        g_j = dds_j.condense(o["f"])
        x_j, _, _ = dd.pcg(dds_j.schur_apply, pre.apply, g_j, 1e-12, 5000)
        Zs.append(x_j)
    for deflate in (False, True):
        x, it, hist, cs = coarse.coarse_pcg(dds.schur_apply, pre.apply, g, np.stack(Zs, axis=1), tol,
                                            5000, deflate=deflate)
        assert cs.spd and cs.k == 3
        assert np.linalg.norm(x - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
        assert it < it_ref
