"""Finite-element layer of the oracle (test infrastructure only; see package doc).

Sec. 1 of the paper states the problem: Hooke's law sigma = 2 mu eps +
lambda tr(eps) I with the Lame constants mu = E/(2(1+nu)),
lambda = nu E/((1+nu)(1-2nu)), clamped and traction boundaries.  Sec. 2
discretises it into K u = f; Sec. 5 (eq. NumberTen) scales each element
stiffness by the element density.  The density exponent p is a parameter
(p = 1 is the paper's variable-thickness sheet, p = 3 the SIMP form used by
the workloads).

Grid conventions (shared only by specification with the GPU library, never by
code): unit elements; 2D node (i, j) has index n = i*(ny+1) + j, 3D node
(i, j, k) has n = (i*(ny+1) + j)*(nz+1) + k; DOF = d*n + c.  Element (ex, ey)
has index ex*ny + ey; 3D element (ex, ey, ez) has (ex*ny + ey)*nz + ez.
"""
import itertools

import numpy as np
import scipy.sparse as sp


# ----------------------------------------------------------------------------
# Material (Sec. 1, Hooke's law and Lame constants)
# ----------------------------------------------------------------------------
def lame(E, nu):
    """Lame constants (mu, lambda_hat) exactly as defined in Sec. 1."""
    if not (E > 0 and -1.0 < nu < 0.5):
        raise ValueError("need E > 0 and -1 < nu < 1/2 (Sec. 1)")
    mu = E / (2.0 * (1.0 + nu))
    lam = nu * E / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


def elasticity_matrix(dim, E, nu, plane_stress=True):
    """Voigt matrix D with sigma = D eps (engineering shear strains).

    3D: isotropic Hooke law of Sec. 1.  Voigt order xx, yy, zz, xy, yz, zx.
    2D plane stress (reading Q2): the same law with sigma_zz = 0, i.e. lambda
    replaced by lambda* = 2 mu lambda / (lambda + 2 mu).  2D plane strain uses
    lambda unchanged.
    """
    mu, lam = lame(E, nu)
    if dim == 3:
        D = np.zeros((6, 6))
        D[:3, :3] = lam
        D[np.arange(3), np.arange(3)] = lam + 2 * mu
        D[3, 3] = D[4, 4] = D[5, 5] = mu
        return D
    if plane_stress:
        lam = 2 * mu * lam / (lam + 2 * mu)
    D = np.array([[lam + 2 * mu, lam, 0.0], [lam, lam + 2 * mu, 0.0], [0.0, 0.0, mu]])
    return D


# ----------------------------------------------------------------------------
# Element stiffness by Gauss quadrature (the FE discretisation of Sec. 2)
# ----------------------------------------------------------------------------
def _ref_nodes(dim):
    """Reference-element node coordinates in {-1, 1}^dim.

    2D order: (-1,-1), (1,-1), (1,1), (-1,1).  3D: the 2D order at zeta=-1,
    then at zeta=+1.
    """
    q = [(-1, -1), (1, -1), (1, 1), (-1, 1)]
    if dim == 2:
        return np.array(q, dtype=float)
    return np.array([(a, b, -1) for a, b in q] + [(a, b, 1) for a, b in q], dtype=float)


def element_node_offsets(dim):
    """Grid offsets of the element's local nodes (same order as _ref_nodes)."""
    return ((_ref_nodes(dim) + 1) / 2).astype(int)


def _shape_grads(dim, xi):
    """Gradients of the multilinear shape functions at reference point xi."""
    nodes = _ref_nodes(dim)
    g = np.zeros((len(nodes), dim))
    for a, na in enumerate(nodes):
        for k in range(dim):
            v = na[k] / 2.0
            for m in range(dim):
                if m != k:
                    v *= (1 + na[m] * xi[m]) / 2.0
            g[a, k] = v
    return g


def strain_matrix(dim, xi, h=1.0):
    """B with eps = B u_e (Sec. 1 linearised strain) at xi, element size h."""
    g = _shape_grads(dim, xi) * (2.0 / h)  # d/dx = (2/h) d/dxi
    nn = len(g)
    if dim == 2:
        B = np.zeros((3, 2 * nn))
        for a in range(nn):
            B[0, 2 * a] = g[a, 0]
            B[1, 2 * a + 1] = g[a, 1]
            B[2, 2 * a] = g[a, 1]
            B[2, 2 * a + 1] = g[a, 0]
        return B
    B = np.zeros((6, 3 * nn))
    for a in range(nn):
        gx, gy, gz = g[a]
        c = 3 * a
        B[0, c] = gx
        B[1, c + 1] = gy
        B[2, c + 2] = gz
        B[3, c], B[3, c + 1] = gy, gx
        B[4, c + 1], B[4, c + 2] = gz, gy
        B[5, c], B[5, c + 2] = gz, gx
    return B


def element_stiffness(dim, E, nu, plane_stress=True, order=3, h=1.0):
    """K_e = integral of B^T D B over the element, Gauss-Legendre of `order`."""
    D = elasticity_matrix(dim, E, nu, plane_stress)
    pts, wts = np.polynomial.legendre.leggauss(order)
    nd = dim * 2 ** dim
    K = np.zeros((nd, nd))
    jac = (h / 2.0) ** dim
    for idx in itertools.product(range(order), repeat=dim):
        xi = np.array([pts[i] for i in idx])
        w = np.prod([wts[i] for i in idx]) * jac
        B = strain_matrix(dim, xi, h)
        K += w * B.T @ D @ B
    return 0.5 * (K + K.T)


def rigid_body_modes(dim, coords):
    """Rigid displacements (translations + infinitesimal rotations) at coords."""
    n = len(coords)
    modes = []
    for c in range(dim):
        m = np.zeros((n, dim))
        m[:, c] = 1.0
        modes.append(m.ravel())
    rots = [(0, 1)] if dim == 2 else [(0, 1), (1, 2), (2, 0)]
    for a, b in rots:
        m = np.zeros((n, dim))
        m[:, a] = -coords[:, b]
        m[:, b] = coords[:, a]
        modes.append(m.ravel())
    return np.array(modes).T


# ----------------------------------------------------------------------------
# Structured grid
# ----------------------------------------------------------------------------
class Grid:
    """Structured grid of unit elements, nx x ny (x nz)."""

    def __init__(self, dim, nx, ny, nz=0):
        self.dim = dim
        self.ne = (nx, ny) if dim == 2 else (nx, ny, nz)
        self.nn = tuple(n + 1 for n in self.ne)
        self.n_nodes = int(np.prod(self.nn))
        self.n_elem = int(np.prod(self.ne))
        self.n_dof = dim * self.n_nodes

    def node_index(self, *ijk):
        n = 0
        for a, nn in zip(ijk, self.nn):
            n = n * nn + a
        return n

    def node_coords(self):
        axes = [np.arange(n) for n in self.nn]
        mesh = np.meshgrid(*axes, indexing="ij")
        return np.stack([m.ravel() for m in mesh], axis=1)

    def element_nodes(self):
        """(n_elem, 2^dim) global node indices, local order of _ref_nodes."""
        axes = [np.arange(n) for n in self.ne]
        mesh = np.meshgrid(*axes, indexing="ij")
        base = [m.ravel() for m in mesh]
        out = np.zeros((self.n_elem, 2 ** self.dim), dtype=np.int64)
        for a, off in enumerate(element_node_offsets(self.dim)):
            out[:, a] = self.node_index(*[b + o for b, o in zip(base, off)])
        return out

    def element_dofs(self):
        en = self.element_nodes()
        d = self.dim
        return (d * en[:, :, None] + np.arange(d)[None, None, :]).reshape(self.n_elem, -1)


def element_factors(rho, E, p):
    """Per-element stiffness factor E * rho_e^p (eq. NumberTen with exponent p)."""
    return E * np.asarray(rho, dtype=float) ** p


def assemble(grid, Ke, factors):
    """Global sparse K = sum_e factor_e P_e^T K_e P_e (CSR, all DOFs)."""
    edofs = grid.element_dofs()
    nd = edofs.shape[1]
    rows = np.repeat(edofs, nd, axis=1).ravel()
    cols = np.tile(edofs, (1, nd)).ravel()
    vals = (factors[:, None] * Ke.ravel()[None, :]).ravel()
    K = sp.coo_matrix((vals, (rows, cols)), shape=(grid.n_dof, grid.n_dof)).tocsr()
    K.sum_duplicates()
    return K


def apply_ebe(grid, Ke, factors, u):
    """Matrix-free K u by the element-by-element definition (any size)."""
    edofs = grid.element_dofs()
    ue = u[edofs]
    ye = (ue @ Ke.T) * factors[:, None]
    y = np.zeros(grid.n_dof)
    np.add.at(y, edofs.ravel(), ye.ravel())
    return y


# ----------------------------------------------------------------------------
# Boundary conditions and loads (Sec. 1 mixed BVP; workload definitions)
# ----------------------------------------------------------------------------
def face_nodes(grid, axis, side):
    """Nodes on the grid face axis=0 (side 0) or axis=n (side 1)."""
    coords = grid.node_coords()
    val = 0 if side == 0 else grid.ne[axis]
    return np.nonzero(coords[:, axis] == val)[0]


def bc_from_spec(grid, spec):
    """Fixed-DOF mask and load vector from a workload BC spec.

    spec keys: "clamp": list of (axis, side) faces with all components fixed;
    "fix": list of (node_ijk, component); "point": list of (node_ijk, force
    vector); "traction": (axis, side, traction vector) applied as consistent
    nodal loads of a uniform surface traction on that face (each boundary
    facet of unit area gives 1/2^(dim-1) of its force to each of its nodes);
    "body": force vector per unit volume, the f of the mixed problem of
    Sec. 1, as consistent nodal loads of the bilinear (trilinear) elements
    (each unit element gives 1/2^dim of its force to each of its nodes).
    """
    d = grid.dim
    fixed = np.zeros(grid.n_dof, dtype=bool)
    f = np.zeros(grid.n_dof)
    for axis, side in spec.get("clamp", []):
        for n in face_nodes(grid, axis, side):
            fixed[d * n:d * n + d] = True
    for ijk, c in spec.get("fix", []):
        fixed[d * grid.node_index(*ijk) + c] = True
    for ijk, force in spec.get("point", []):
        n = grid.node_index(*ijk)
        f[d * n:d * n + d] += np.asarray(force, dtype=float)
    if "traction" in spec:
        axis, side, t = spec["traction"]
        t = np.asarray(t, dtype=float)
        others = [a for a in range(d) if a != axis]
        val = 0 if side == 0 else grid.ne[axis]
        ranges = [range(grid.ne[a]) for a in others]
        share = 1.0 / 2 ** (d - 1)
        for cell in itertools.product(*ranges):
            for corner in itertools.product((0, 1), repeat=d - 1):
                ijk = [0] * d
                ijk[axis] = val
                for a, c0, o in zip(others, cell, corner):
                    ijk[a] = c0 + o
                n = grid.node_index(*ijk)
                f[d * n:d * n + d] += share * t
    if "body" in spec:
        b = np.asarray(spec["body"], dtype=float)
        en = grid.element_nodes()
        share = 1.0 / 2 ** d
        for a in range(en.shape[1]):
            for c in range(d):
                np.add.at(f, d * en[:, a] + c, share * b[c])
    f[fixed] = 0.0
    return fixed, f
