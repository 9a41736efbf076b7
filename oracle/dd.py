"""Domain-decomposition layer of the oracle (test infrastructure only).

Follows the paper's Sec. 1-3 in its own notation:

* Sec. 1: N non-overlapping subdomains Omega_i; skeleton Gamma; interior set I.
  Discrete reading (Q11): a node is on Gamma iff it lies in the closure of two
  or more subdomains; Dirichlet (clamped) DOFs are eliminated everywhere.
* Sec. 2, eq. NumberFour / NumberFive: K = [[K_II, K_IG], [K_GI, K_GG]] with
  K_II the direct sum of the subdomain blocks K_{I_i I_i}.
* Sec. 2, eq. 3MatSplit2: K_{I_iI_i} u1_i = f_{I_i};  S u_G = f_G - sum_i
  K_{G I_i} u1_i;  K_{I_iI_i} u2_i = -K_{I_i G} u_G;  u = (u1 + u2, u_G).
* Sec. 3, eq. NumberEight / NumberNine: H_theta = M + M (M^-1 L)^(1-theta),
  its spectrally equivalent form Htilde_theta = M (M^-1 L)^(1-theta), applied
  component-wise.  Sec. 4 builds the parallel preconditioner from the
  interface operators restricted to each Gamma_i with the cross points
  removed; the hot path uses exactly that face-local form as S~ (reading Q6),
  with a diagonal at the cross points (Q7) and a per-face scale (Q8).
* The interface Krylov method is PCG on S u_G = g (reading Q4, stopping test
  Q12); `pcg_relaxed` is its mixed-precision form (the paper is silent on
  precision below its double).
"""
import itertools

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import fem


class Decomposition:
    """DOF classification for a structured grid split into sub^dim blocks."""

    def __init__(self, grid, sub, fixed):
        self.grid = grid
        self.sub = sub
        d = grid.dim
        for n in grid.ne:
            if n % sub:
                raise ValueError("subdomain edge must divide the grid")
        self.nsub_axis = tuple(n // sub for n in grid.ne)
        self.n_sub = int(np.prod(self.nsub_axis))
        self.fixed = np.asarray(fixed, dtype=bool)
        coords = grid.node_coords()
        # subdomain candidates per axis for every node (closure membership)
        self.node_subs = []
        for n in range(grid.n_nodes):
            per_axis = []
            for a in range(d):
                x = coords[n, a]
                cands = [q for q in (x // sub - 1, x // sub)
                         if 0 <= q < self.nsub_axis[a] and q * sub <= x <= (q + 1) * sub]
                per_axis.append(sorted(set(cands)))
            subs = [self.sub_index(*c) for c in itertools.product(*per_axis)]
            self.node_subs.append(frozenset(subs))
        self.gamma_node = np.array([len(s) >= 2 for s in self.node_subs])
        free = ~self.fixed
        dof_node = np.arange(grid.n_dof) // d
        self.gamma_dofs = np.nonzero(free & self.gamma_node[dof_node])[0]
        self.interior_dofs = []  # per subdomain, sorted global DOFs
        owner = np.full(grid.n_nodes, -1)
        for n, s in enumerate(self.node_subs):
            if len(s) == 1:
                owner[n] = next(iter(s))
        for i in range(self.n_sub):
            nodes = np.nonzero(owner == i)[0]
            dofs = (d * nodes[:, None] + np.arange(d)[None, :]).ravel()
            self.interior_dofs.append(np.sort(dofs[free[dofs]]))
        self.all_interior = np.concatenate(self.interior_dofs)

    def sub_index(self, *q):
        n = 0
        for a, na in zip(q, self.nsub_axis):
            n = n * na + a
        return n

    def sub_elements(self, i):
        """Element indices of subdomain i."""
        q = []
        r = i
        for na in reversed(self.nsub_axis):
            q.append(r % na)
            r //= na
        q = q[::-1]
        ranges = [range(qa * self.sub, (qa + 1) * self.sub) for qa in q]
        out = []
        for e in itertools.product(*ranges):
            idx = 0
            for a, n in zip(e, self.grid.ne):
                idx = idx * n + a
            out.append(idx)
        return np.array(out)


class DDSystem:
    """Block partition of K (eq. NumberFour/NumberFive) and the 3-step solve."""

    def __init__(self, dec, K):
        self.dec = dec
        self.K = K.tocsr()
        G = dec.gamma_dofs
        self.K_GG = self.K[G][:, G].tocsr()
        self.blocks = []  # per subdomain: (I dofs, cho factor of K_IiIi, K_{I_i G})
        for I in dec.interior_dofs:
            KII = self.K[I][:, I].toarray()
            cf = sla.cho_factor(KII, lower=True)
            KIG = self.K[I][:, G].tocsr()
            self.blocks.append((I, cf, KIG))

    def solve_II(self, b_I_list):
        """Block-diagonal K_II^-1 (eq. NumberFive): one solve per subdomain."""
        return [sla.cho_solve(cf, b) for (I, cf, _), b in zip(self.blocks, b_I_list)]

    def schur_apply(self, x, pool=None):
        """S x = K_GG x - sum_i K_{G I_i} K_{I_i I_i}^-1 K_{I_i G} x (eq. 3MatSplit).

        pool: an optional concurrent.futures executor that computes the
        subdomain terms K_{G I_i} K_{I_i I_i}^-1 K_{I_i G} x side by side (the
        subdomains are independent, Sec. 2); they are still subtracted in
        subdomain order, so the result is bitwise the serial one.
        """
        y = self.K_GG @ x

        def term(blk):
            I, cf, KIG = blk
            return KIG.T @ sla.cho_solve(cf, KIG @ x)

        terms = map(term, self.blocks) if pool is None else pool.map(term, self.blocks)
        for t in terms:
            y -= t
        return y

    def schur_dense(self):
        """Explicit S (small grids only)."""
        S = self.K_GG.toarray()
        for I, cf, KIG in self.blocks:
            W = sla.cho_solve(cf, KIG.toarray())
            S -= KIG.T.toarray() @ W
        return 0.5 * (S + S.T)

    def condense(self, f):
        """g = f_G - sum_i K_{G I_i} K_{I_i I_i}^-1 f_{I_i} (eq. 3MatSplit2, 2nd line)."""
        g = f[self.dec.gamma_dofs].copy()
        for I, cf, KIG in self.blocks:
            u1 = sla.cho_solve(cf, f[I])
            g -= KIG.T @ u1
        return g

    def back_substitute(self, f, uG):
        """u_I = K_II^-1 (f_I - K_IG u_G); assemble u (eq. 3MatSplit2, 1st+3rd line)."""
        u = np.zeros(self.K.shape[0])
        u[self.dec.gamma_dofs] = uG
        for I, cf, KIG in self.blocks:
            u[I] = sla.cho_solve(cf, f[I] - KIG @ uG)
        return u


# ----------------------------------------------------------------------------
# Interface preconditioner (Sec. 3 eq. NumberEight/NumberNine; Sec. 4)
# ----------------------------------------------------------------------------
def interface_mass_laplacian(dec):
    """Mass M and Laplacian L assembled on the skeleton Gamma (scalar, per node).

    Gamma is meshed by the element edges (2D) / element faces (3D) that lie on
    it: a facet whose nodes' subdomain sets share two or more subdomains.
    Returns (M, L) as sparse matrices over all grid nodes (zero off Gamma).
    """
    grid = dec.grid
    d = grid.dim
    nn = grid.n_nodes
    rows, cols, mv, lv = [], [], [], []
    if d == 2:
        Me = np.array([[2.0, 1.0], [1.0, 2.0]]) / 6.0
        Le = np.array([[1.0, -1.0], [-1.0, 1.0]])
        facets = []
        nx, ny = grid.ne
        for i in range(nx + 1):
            for j in range(ny + 1):
                n0 = grid.node_index(i, j)
                if i < nx:
                    facets.append((n0, grid.node_index(i + 1, j)))
                if j < ny:
                    facets.append((n0, grid.node_index(i, j + 1)))
    else:
        # bilinear quad on a unit square: scalar mass and Laplacian by Gauss 3x3
        pts, wts = np.polynomial.legendre.leggauss(3)
        ref = np.array([(-1, -1), (1, -1), (1, 1), (-1, 1)], float)
        Me = np.zeros((4, 4))
        Le = np.zeros((4, 4))
        for a in range(3):
            for b in range(3):
                xi = np.array([pts[a], pts[b]])
                w = wts[a] * wts[b] * 0.25
                N = np.array([(1 + r[0] * xi[0]) * (1 + r[1] * xi[1]) / 4 for r in ref])
                dN = np.array([[r[0] * (1 + r[1] * xi[1]) / 4, r[1] * (1 + r[0] * xi[0]) / 4]
                               for r in ref]) * 2.0
                Me += w * np.outer(N, N)
                Le += w * dN @ dN.T
        facets = []
        ne = grid.ne
        for axis in range(3):
            o = [a for a in range(3) if a != axis]
            for x in range(grid.nn[axis]):
                for c0 in range(ne[o[0]]):
                    for c1 in range(ne[o[1]]):
                        quad = []
                        for d0, d1 in ((0, 0), (1, 0), (1, 1), (0, 1)):
                            ijk = [0, 0, 0]
                            ijk[axis] = x
                            ijk[o[0]] = c0 + d0
                            ijk[o[1]] = c1 + d1
                            quad.append(grid.node_index(*ijk))
                        facets.append(tuple(quad))
    for fct in facets:
        common = frozenset.intersection(*[dec.node_subs[n] for n in fct])
        if len(common) < 2:
            continue
        for a, na in enumerate(fct):
            for b, nb in enumerate(fct):
                rows.append(na)
                cols.append(nb)
                mv.append(Me[a, b])
                lv.append(Le[a, b])
    M = sp.coo_matrix((mv, (rows, cols)), shape=(nn, nn)).tocsr()
    L = sp.coo_matrix((lv, (rows, cols)), shape=(nn, nn)).tocsr()
    return M, L


class FaceBlock:
    """One (face, component) block of the face-local preconditioner."""

    def __init__(self, dofs, M, L, theta):
        self.dofs = dofs  # positions in the Gamma vector
        self.M = M
        self.L = L
        mu, V = sla.eigh(L, M)  # L V = M V diag(mu), V^T M V = I (Sec. 3)
        self.mu = mu
        self.V = V
        self.singular = mu[0] <= 1e-12 * max(mu[-1], 1.0)
        if self.singular:
            # Q5: the L-only form is singular (face with no removed end);
            # use H_theta = M + M (M^-1 L)^(1-theta) of eq. NumberEight.  The
            # kernel of L_f is exact (constants), so eigenvalues at rounding
            # level are zero; the fractional power would amplify their noise.
            mu0 = np.where(mu <= 1e-12 * max(mu[-1], 1.0), 0.0, mu)
            lam = 1.0 + mu0 ** (1.0 - theta)
        else:
            lam = mu ** (1.0 - theta)  # Htilde_theta = M V diag(mu^(1-theta)) V^T M
        self.H = M @ V @ np.diag(lam) @ V.T @ M  # the face norm matrix itself
        self.Hinv = V @ np.diag(1.0 / lam) @ V.T  # = H^-1 since V^T M V = I
        self.alpha = 1.0


class FacePreconditioner:
    """z = S~^-1 r: face-local Htilde_theta^-1 per component, diagonal at cross points.

    S~ is block diagonal over (face, component) blocks (eq. NumberNine applied
    on each face Gamma_i with the cross points removed, Sec. 4) plus the
    diagonal of K_GG at cross-point / wirebasket DOFs (reading Q7).  Scaling
    of each face block against the material (reading Q8; the paper's tests are
    homogeneous and it gives none):
      face_scaling="dof" (default): S~_f = W H_f W with the diagonal
        W = diag(sqrt(diag(K_GG)_i / diag(H_f)_i)), so diag(S~_f) = diag(K_GG)
        on the face (close to the scalar scaling below on a homogeneous
        face, where only diag(H_f) varies, near the face ends);
      face_scaling="face" (or True): S~_f = alpha H_f with alpha =
        mean(diag K_GG over the block) / mean(diag H_f);
      face_scaling=False: S~_f = H_f (paper-literal).
    crosspoint="identity" is the paper-literal alternative of Q7.
    """

    def __init__(self, dec, K, theta=0.5, face_scaling="dof", crosspoint="diag"):
        self.dec = dec
        grid = dec.grid
        d = grid.dim
        G = dec.gamma_dofs
        pos = {int(g): k for k, g in enumerate(G)}
        M, L = interface_mass_laplacian(dec)
        Kdiag = K.diagonal()
        faces = {}
        self.cross_pos = []
        for k, g in enumerate(G):
            n = int(g) // d
            subs = dec.node_subs[n]
            if len(subs) == 2:
                faces.setdefault((subs, int(g) % d), []).append(n)
            else:
                self.cross_pos.append(k)
        self.blocks = []
        for (subs, c), nodes in sorted(faces.items(), key=lambda kv: (sorted(kv[0][0]), kv[0][1])):
            nodes = np.array(sorted(nodes))
            Mf = M[nodes][:, nodes].toarray()
            Lf = L[nodes][:, nodes].toarray()
            fb = FaceBlock(np.array([pos[d * n + c] for n in nodes]), Mf, Lf, theta)
            kd = Kdiag[G[fb.dofs]]
            fb.w = np.ones(len(fb.dofs))  # S~_f^-1 = W^-1 H_f^-1 W^-1 / alpha
            if face_scaling == "dof":
                fb.w = np.sqrt(kd / np.diag(fb.H))
            elif face_scaling:
                fb.alpha = kd.mean() / np.diag(fb.H).mean()
            self.blocks.append(fb)
        self.cross_pos = np.array(self.cross_pos, dtype=np.int64)
        if crosspoint == "diag":
            self.cross_scale = 1.0 / Kdiag[G[self.cross_pos]]
        else:
            self.cross_scale = np.ones(len(self.cross_pos))

    def apply(self, r):
        z = np.zeros_like(r)
        for fb in self.blocks:
            z[fb.dofs] = (fb.Hinv @ (r[fb.dofs] / fb.w)) / (fb.w * fb.alpha)
        z[self.cross_pos] = r[self.cross_pos] * self.cross_scale
        return z

    def dense(self):
        """S~^-1 as a dense matrix (small grids)."""
        n = len(self.dec.gamma_dofs)
        P = np.zeros((n, n))
        for fb in self.blocks:
            Wi = np.diag(1.0 / fb.w)
            P[np.ix_(fb.dofs, fb.dofs)] = Wi @ fb.Hinv @ Wi / fb.alpha
        P[self.cross_pos, self.cross_pos] = self.cross_scale
        return P


# ----------------------------------------------------------------------------
# Interface PCG (reading Q4) and the full DD solve (eq. 3MatSplit2)
# ----------------------------------------------------------------------------
def pcg(apply_S, apply_P, g, tol, max_it, x0=None, ref_norm=None):
    """Preconditioned CG on S x = g.

    Stops when ||r||_2 <= tol * ref_norm (ref_norm defaults to ||g||_2,
    reading Q12).  Returns (x, iterations, history of ||r||_2).  The iteration
    count is the number of S applications after the initial residual.
    """
    x = np.zeros_like(g) if x0 is None else x0.copy()
    r = g - apply_S(x) if x0 is not None else g.copy()
    ref = np.linalg.norm(g) if ref_norm is None else ref_norm
    hist = [np.linalg.norm(r)]
    if hist[-1] <= tol * ref:
        return x, 0, hist
    z = apply_P(r)
    p = z.copy()
    rz = r @ z
    it = 0
    while it < max_it:
        q = apply_S(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        hist.append(np.linalg.norm(r))
        if hist[-1] <= tol * ref:
            break
        z = apply_P(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, hist


def pcg_relaxed(apply_S, apply_S_lo, apply_P, g, tol, max_it, switch, delta=0.1, check_every=1,
                ref_norm=None):
    """PCG on S x = g that switches to a cheaper, less accurate operator S_lo
    once the residual is small, and stops only on the true residual.

    The paper fixes no precision below its MATLAB double; this is the mixed
    form of the interface solve (FP64 Schur complements early, a low-precision
    copy late), built from two published results:
      * relaxation in inexact Krylov methods (Bouras & Fraysse 2005; van den
        Eshof & Sleijpen 2004): the error allowed in the operator grows as the
        residual falls, so S is applied until ||r|| <= switch * ref_norm and
        S_lo from then on;
      * reliable updates (Sleijpen & van der Vorst 1996): after the switch,
        whenever the recursive residual has fallen below delta times its
        largest value since the last replacement, or below the tolerance, it
        is replaced by the true residual g - S x computed with S; the search
        direction is kept, so the Krylov space is not restarted.
    The decisions (switch, replacement, stop) are taken every check_every
    iterations and whenever the recursive residual meets the tolerance.  In
    the S phase the stopping test is the textbook one; in the S_lo phase the
    iteration stops only after a replacement shows ||g - S x|| <= tol *
    ref_norm.  With switch = 0 and check_every = 1 this is `pcg` operation for
    operation.

    Returns (x, iterations, iterations with S_lo, replacements, history of
    ||r||_2 after each iteration)."""
    x = np.zeros_like(g)
    r = g.copy()
    ref = np.linalg.norm(g) if ref_norm is None else ref_norm
    hist = [np.linalg.norm(r)]
    if hist[-1] <= tol * ref:
        return x, 0, 0, 0, hist
    z = apply_P(r)
    p = z.copy()
    rz = r @ z
    lo = False
    r_max = hist[-1]
    it = n_lo = n_true = 0
    while it < max_it:
        q = (apply_S_lo if lo else apply_S)(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        n_lo += lo
        rn = np.linalg.norm(r)
        if it % check_every == 0 or rn <= tol * ref:
            if not lo and rn <= tol * ref:
                hist.append(rn)
                break
            if not lo and rn <= switch * ref:
                lo = True
                r_max = rn
            elif lo and (rn < delta * r_max or rn <= tol * ref):
                r = g - apply_S(x)
                n_true += 1
                rn = np.linalg.norm(r)
                r_max = rn
                if rn <= tol * ref:
                    hist.append(rn)
                    break
            r_max = max(r_max, rn)
        hist.append(rn)
        z = apply_P(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, n_lo, n_true, hist


def dd_solve(dd, precond, f, tol=1e-12, max_it=5000, ref="f"):
    """Three-step DD solve of eq. 3MatSplit2 with interface PCG.

    ref="f": PCG stops at ||r_G|| <= tol ||f|| (the global relative residual
    of the assembled u, since the interior equations are solved exactly);
    ref="g": stops at ||r_G|| <= tol ||g|| (Q12's interface form).
    """
    g = dd.condense(f)
    ref_norm = np.linalg.norm(f) if ref == "f" else np.linalg.norm(g)
    uG, it, hist = pcg(dd.schur_apply, precond.apply, g, tol, max_it, ref_norm=ref_norm)
    u = dd.back_substitute(f, uG)
    return u, it, hist


def build(grid, sub, fixed, Ke, factors):
    """Convenience: decomposition, global K (all DOFs) and its DD system."""
    dec = Decomposition(grid, sub, fixed)
    K = fem.assemble(grid, Ke, factors)
    free = ~dec.fixed
    # eliminate clamped DOFs: zero their rows/cols, unit diagonal
    D = sp.diags(free.astype(float))
    Kr = (D @ K @ D + sp.diags((~free).astype(float))).tocsr()
    return dec, Kr, DDSystem(dec, Kr)
