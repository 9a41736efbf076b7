"""Pins of the oracle's relaxed mixed-precision PCG (`dd.pcg_relaxed`).

Independent checks: with no switch it is the textbook PCG operation for
operation; with an exact "low" operator the replacements change nothing but
rounding; with the Schur complement rounded to FP32 -- where PCG on that
operator alone stalls far above the tolerance in the true residual -- it
still stops on a true FP64 residual below the tolerance, because it
replaces the recursive residual with g - S x computed with S (reliable
updates), and it keeps the FP64 iteration count within a few per cent
(relaxation: the operator's error only enters once the residual is small).
"""
import numpy as np
import pytest

from oracle import dd, fem
import workloads


def _interface(nx, ny, sub, seed, theta=0.5):
    cfg = workloads.small_config(nx, ny, sub, seed=seed)
    grid = fem.Grid(2, nx, ny)
    fixed, f = fem.bc_from_spec(grid, cfg["bc"])
    Ke = fem.element_stiffness(2, cfg["E"], cfg["nu"])
    fac = fem.element_factors(workloads.density(cfg), cfg["E"], cfg["p"])
    dec, K, dds = dd.build(grid, sub, fixed, Ke, fac)
    pre = dd.FacePreconditioner(dec, K, theta=theta)
    S = dds.schur_dense()
    return S, pre.apply, dds.condense(f), np.linalg.norm(f)


@pytest.fixture(scope="module")
def grf_64x32():
    # 64x32 cantilever, 8 subdomains of 16x16, GRF densities in [1e-3, 1], p = 3
    return _interface(64, 32, 16, seed=3)


@pytest.fixture(scope="module")
def grf_128x64():
    # 128x64 cantilever, 32 subdomains of 16x16 (1636 interface DOFs), GRF
    # densities in [1e-3, 1], p = 3: a stiffness contrast of 1e9
    return _interface(128, 64, 16, seed=3)


def test_without_a_switch_it_is_textbook_pcg(grf_64x32):
    S, P, g, fn = grf_64x32
    x0, it0, h0 = dd.pcg(lambda v: S @ v, P, g, 1e-10, 5000, ref_norm=fn)
    x1, it1, n_lo, n_true, h1 = dd.pcg_relaxed(lambda v: S @ v, None, P, g, 1e-10, 5000, switch=0.0,
                                               ref_norm=fn)
    assert it1 == it0 and n_lo == 0 and n_true == 0
    assert np.array_equal(x1, x0) and h1 == h0


def test_exact_low_operator_changes_only_rounding(grf_64x32):
    S, P, g, fn = grf_64x32
    A = lambda v: S @ v
    x0, it0, _ = dd.pcg(A, P, g, 1e-10, 5000, ref_norm=fn)
    x1, it1, n_lo, n_true, _ = dd.pcg_relaxed(A, A, P, g, 1e-10, 5000, switch=1e-2, delta=0.1,
                                              check_every=4, ref_norm=fn)
    assert n_lo > 0 and n_true >= 1
    assert abs(it1 - it0) <= 4  # decisions every 4 iterations
    assert np.linalg.norm(x1 - x0) <= 1e-8 * np.linalg.norm(x0)


def test_fp32_schur_complement_reaches_the_fp64_tolerance(grf_128x64):
    S, P, g, fn = grf_128x64
    tol = 1e-8
    S32 = S.astype(np.float32)
    A = lambda v: S @ v
    A_lo = lambda v: (S32 @ v.astype(np.float32)).astype(np.float64)
    true = lambda x: np.linalg.norm(g - A(x)) / fn
    # the case discriminates: PCG on the FP32 operator alone meets the
    # tolerance in its recursive residual but not in the true one
    x_lo, _, h_lo = dd.pcg(A_lo, P, g, tol, 20000, ref_norm=fn)
    assert h_lo[-1] <= tol * fn and true(x_lo) > 30 * tol
    x64, it64, _ = dd.pcg(A, P, g, tol, 20000, ref_norm=fn)
    for switch in (1e-1, 1e-2, 1e-3):
        x, it, n_lo, n_true, hist = dd.pcg_relaxed(A, A_lo, P, g, tol, 20000, switch=switch, delta=0.1,
                                                   check_every=4, ref_norm=fn)
        assert true(x) <= tol and hist[-1] == pytest.approx(true(x) * fn, rel=1e-12)
        assert n_lo >= 0.15 * it and n_true >= 1
        assert it <= 1.05 * it64 + 4
        assert np.linalg.norm(x - x64) <= 1e-6 * np.linalg.norm(x64)


def test_replacement_uses_the_accurate_operator(grf_128x64):
    # a planted mistake: replacing the residual with the low operator as well
    # leaves the iteration blind to its drift, and the true residual misses
    # the tolerance -- what the replacement with S prevents
    S, P, g, fn = grf_128x64
    tol = 1e-8
    S32 = S.astype(np.float32)
    A_lo = lambda v: (S32 @ v.astype(np.float32)).astype(np.float64)
    # (its own residual g - S_lo x has an FP32 rounding floor above the
    # tolerance, so it runs to max_it: twice the FP64 count here)
    x, it, *_ = dd.pcg_relaxed(A_lo, A_lo, P, g, tol, 400, switch=1.0, delta=0.1, ref_norm=fn)
    assert np.linalg.norm(g - S @ x) / fn > 30 * tol
