"""Pins of the oracle's finite-element layer against independent mathematics.

Each test checks the oracle against something other than itself: an exact
symbolic integration, textbook identities of isotropic elasticity, rigid-body
invariance, the linear-field patch test, and load totals.
"""
import numpy as np
import pytest

from oracle import dd, direct, fem
from workloads import cantilever_3d


def test_lame_textbook_identities():
    # Sec. 1 defines mu, lambda from E, nu; the inverse relations of isotropic
    # elasticity must give E and nu back.
    for E, nu in [(1.0, 0.3), (210.0, 0.25), (3.0, -0.5), (1.0, 0.49)]:
        mu, lam = fem.lame(E, nu)
        assert np.isclose(mu * (3 * lam + 2 * mu) / (lam + mu), E, rtol=1e-14)
        assert np.isclose(lam / (2 * (lam + mu)), nu, rtol=1e-13, atol=1e-15)


def test_lame_rejects_out_of_range():
    for nu in (0.5, -1.0, 0.7):
        with pytest.raises(ValueError):
            fem.lame(1.0, nu)
    with pytest.raises(ValueError):
        fem.lame(0.0, 0.3)


def test_plane_stress_from_3d_compliance():
    # Independent route (reading Q2): invert the in-plane block of the 3D
    # compliance with sigma_zz = 0: eps_xx = (s_xx - nu s_yy)/E, gamma = s_xy/G.
    for E, nu in [(1.0, 0.3), (5.0, 0.1), (1.0, 0.45)]:
        G = E / (2 * (1 + nu))
        C = np.array([[1 / E, -nu / E, 0], [-nu / E, 1 / E, 0], [0, 0, 1 / G]])
        assert np.allclose(fem.elasticity_matrix(2, E, nu, True), np.linalg.inv(C), rtol=1e-13)
        # 3D: D must invert the full 6x6 compliance
        C3 = np.zeros((6, 6))
        C3[:3, :3] = -nu / E
        C3[np.arange(3), np.arange(3)] = 1 / E
        C3[3, 3] = C3[4, 4] = C3[5, 5] = 1 / G
        assert np.allclose(fem.elasticity_matrix(3, E, nu), np.linalg.inv(C3), rtol=1e-12)


def test_q1_stiffness_exact_symbolic():
    # Exact integration with sympy on [0,1]^2, shape functions written directly
    # in physical coordinates, D from the compliance inverse: an independent
    # derivation of the unit-square plane-stress element (node order
    # (0,0),(1,0),(1,1),(0,1), DOFs interleaved).
    sympy = pytest.importorskip("sympy")
    x, y = sympy.symbols("x y")
    E, nu = sympy.Rational(1), sympy.Rational(3, 10)
    N = [(1 - x) * (1 - y), x * (1 - y), x * y, (1 - x) * y]
    B = sympy.zeros(3, 8)
    for a, Na in enumerate(N):
        B[0, 2 * a] = sympy.diff(Na, x)
        B[1, 2 * a + 1] = sympy.diff(Na, y)
        B[2, 2 * a] = sympy.diff(Na, y)
        B[2, 2 * a + 1] = sympy.diff(Na, x)
    G = E / (2 * (1 + nu))
    C = sympy.Matrix([[1 / E, -nu / E, 0], [-nu / E, 1 / E, 0], [0, 0, 1 / G]])
    D = C.inv()
    integrand = B.T * D * B
    K = integrand.applyfunc(lambda v: sympy.integrate(v, (x, 0, 1), (y, 0, 1)))
    Kexact = np.array(K.evalf(30).tolist(), dtype=float)
    for order in (2, 3):
        Ko = fem.element_stiffness(2, 1.0, 0.3, True, order=order)
        assert np.allclose(Ko, Kexact, rtol=0, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_element_rigid_modes_and_rank(dim):
    Ke = fem.element_stiffness(dim, 1.0, 0.3)
    assert np.allclose(Ke, Ke.T, atol=0)
    w = np.linalg.eigvalsh(Ke)
    nzero = 3 if dim == 2 else 6
    assert np.all(w[:nzero] < 1e-13 * w[-1])
    assert np.all(w[nzero:] > 1e-6 * w[-1])
    R = fem.rigid_body_modes(dim, fem.element_node_offsets(dim).astype(float))
    assert np.abs(Ke @ R).max() < 1e-14 * np.abs(Ke).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_gauss_orders_agree(dim):
    # bilinear/trilinear products are integrated exactly by 2-point Gauss
    K2 = fem.element_stiffness(dim, 1.0, 0.3, order=2)
    K3 = fem.element_stiffness(dim, 1.0, 0.3, order=3)
    assert np.abs(K2 - K3).max() < 1e-14 * np.abs(K3).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_strain_energy(dim):
    # A linear field u = A x has constant strain eps; its element energy is
    # eps^T D eps times the unit volume.
    rng = np.random.default_rng(5)
    A = rng.standard_normal((dim, dim))
    X = fem.element_node_offsets(dim).astype(float)
    u = (X @ A.T).ravel()
    if dim == 2:
        eps = np.array([A[0, 0], A[1, 1], A[0, 1] + A[1, 0]])
    else:
        eps = np.array([A[0, 0], A[1, 1], A[2, 2], A[0, 1] + A[1, 0],
                        A[1, 2] + A[2, 1], A[2, 0] + A[0, 2]])
    D = fem.elasticity_matrix(dim, 2.0, 0.27)
    Ke = fem.element_stiffness(dim, 2.0, 0.27)
    assert np.isclose(u @ Ke @ u, eps @ D @ eps, rtol=1e-13)


def test_floating_subdomain_rigid_modes():
    # Neumann (floating) stiffness of one subdomain annihilates rigid motions
    # for any positive densities.
    grid = fem.Grid(2, 8, 8)
    Ke = fem.element_stiffness(2, 1.0, 0.3)
    rho = np.random.default_rng(1).uniform(1e-3, 1.0, grid.n_elem)
    K = fem.assemble(grid, Ke, fem.element_factors(rho, 1.0, 3.0))
    R = fem.rigid_body_modes(2, grid.node_coords().astype(float))
    assert np.abs(K @ R).max() <= 1e-13 * abs(K).max() * np.abs(R).max()


def test_ebe_equals_assembled():
    grid = fem.Grid(3, 4, 3, 2)
    Ke = fem.element_stiffness(3, 1.0, 0.3)
    rng = np.random.default_rng(2)
    fac = rng.uniform(0.1, 1.0, grid.n_elem)
    u = rng.standard_normal(grid.n_dof)
    K = fem.assemble(grid, Ke, fac)
    assert np.allclose(K @ u, fem.apply_ebe(grid, Ke, fac, u), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("dim,ne,sub", [(2, (12, 8), 4), (3, (4, 4, 4), 2)])
def test_patch_test_dd(dim, ne, sub):
    # Linear displacement prescribed on the whole outer boundary, uniform
    # material: the DD three-step solve must reproduce the linear field at
    # every interior node (Q1/H8 pass the patch test exactly).
    grid = fem.Grid(dim, *ne)
    rng = np.random.default_rng(3)
    a = rng.standard_normal(dim)
    A = rng.standard_normal((dim, dim))
    X = grid.node_coords().astype(float)
    u_lin = (a[None, :] + X @ A.T).ravel()
    fixed = np.zeros(grid.n_dof, dtype=bool)
    for axis in range(dim):
        for side in (0, 1):
            for n in fem.face_nodes(grid, axis, side):
                fixed[dim * n:dim * n + dim] = True
    Ke = fem.element_stiffness(dim, 1.0, 0.3)
    fac = np.full(grid.n_elem, 0.7)
    K = fem.assemble(grid, Ke, fac)
    # lift the prescribed values: free rows get f = -K_fd u_d
    f = -(K @ np.where(fixed, u_lin, 0.0))
    f[fixed] = 0.0
    dec, Kr, dds = dd.build(grid, sub, fixed, Ke, fac)
    pre = dd.FacePreconditioner(dec, Kr)
    u, it, _ = dd.dd_solve(dds, pre, f, tol=1e-14)
    u = np.where(fixed, u_lin, u)
    assert np.abs(u - u_lin).max() < 1e-11 * np.abs(u_lin).max()


def test_traction_total_force_3d():
    grid = fem.Grid(3, 6, 4, 2)
    fixed, f = fem.bc_from_spec(grid, cantilever_3d(6, 4, 2))
    fz = f[2::3]
    assert np.isclose(fz.sum(), -1.0, rtol=1e-14)
    assert np.allclose(f[0::3], 0) and np.allclose(f[1::3], 0)
    # interior nodes of the loaded face carry 4 quarter shares
    n = grid.node_index(6, 2, 1)
    assert np.isclose(f[3 * n + 2], -1.0 / 8)
    assert fixed.sum() == 3 * 5 * 3


def test_direct_solver_against_dense():
    grid = fem.Grid(2, 6, 4)
    Ke = fem.element_stiffness(2, 1.0, 0.3)
    rho = np.random.default_rng(4).uniform(1e-3, 1, grid.n_elem)
    K = fem.assemble(grid, Ke, fem.element_factors(rho, 1.0, 3.0))
    fixed, f = fem.bc_from_spec(grid, {"clamp": [(0, 0)], "point": [((6, 2), (0.0, -1.0))]})
    u = direct.solve(K, f, fixed)
    free = ~fixed
    ud = np.linalg.solve(K.toarray()[np.ix_(free, free)], f[free])
    assert np.allclose(u[free], ud, rtol=1e-9, atol=0)
    assert direct.rel_residual(K, f, u, fixed) < 1e-13


@pytest.mark.parametrize("dim,ne", [(2, (6, 4)), (3, (3, 2, 2))])
def test_body_force_loads_are_work_equivalent(dim, ne):
    # consistent nodal loads of a uniform body force b: for any linear field
    # u(x) = a + B x (interpolated exactly by the bilinear/trilinear elements)
    # f^T u equals the integral of b . u over the unit-element grid, a closed
    # form: b . (a V + B c V) with V the volume and c the centroid
    grid = fem.Grid(dim, *ne)
    b = np.arange(1.0, dim + 1.0) * np.array([1.0, -0.75, 0.5][:dim])
    _, f = fem.bc_from_spec(grid, {"body": tuple(b)})
    rng = np.random.default_rng(8)
    a = rng.standard_normal(dim)
    B = rng.standard_normal((dim, dim))
    X = grid.node_coords().astype(float)
    u = (a[None, :] + X @ B.T).ravel()
    V = float(np.prod(ne))
    c = np.array(ne, dtype=float) / 2.0
    assert abs(f @ u - b @ (a * V + B @ c * V)) <= 1e-12 * V * np.abs(b).sum() * (1 + np.abs(B).sum())
    # an interior node carries exactly b (2^dim elements, 1/2^dim each)
    inner = grid.node_index(*[1] * dim)
    assert np.allclose(f[dim * inner:dim * inner + dim], b, rtol=1e-15, atol=0)

