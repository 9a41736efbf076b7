"""Global-interface preconditioner of Sec. 3 (test infrastructure only).

eq. NumberEight/NumberNine on the whole skeleton Gamma (the form used for the
paper's Tables 1-3), as opposed to the face-local form of Sec. 4 in
`dd.FacePreconditioner`: for each displacement component,

    Htilde_theta = M (M^-1 L)^(1 - theta),

M and L the scalar mass and Laplacian assembled on Gamma
(`dd.interface_mass_laplacian`) restricted to that component's free Gamma
nodes.  With the generalised eigenpairs L V = M V diag(mu), V^T M V = I,
Htilde_theta^-1 = V diag(mu^(theta - 1)) V^T.  Where L restricted to the free
nodes is singular (a part of Gamma that touches no clamped node), reading Q5
applies: H_theta = M + M (M^-1 L)^(1 - theta), i.e. 1 + mu^(1 - theta).

Two ways to apply S~^-1 r:
  * exactly, from the eigendecomposition (small grids; the paper notes its
    O(n_Gamma^3) cost);
  * by inverse Lanczos (Sec. 3, after Arioli and Loghin): k steps of Lanczos
    for B = L^-1 M in the M inner product from b = M^-1 r give B Q_k ~ Q_k T_k,
    and Htilde^-1 r = (M^-1 L)^(theta - 1) b = B^(1 - theta) b
    ~ ||b||_M Q_k T_k^(1 - theta) e_1.  Each step solves with L (here by a
    sparse direct factorisation; the paper uses an inner PCG).  The result
    depends nonlinearly on r for k below the dimension, hence flexible GMRES
    outside (`fgmres`).
Both act on the Gamma vector in the decomposition's Gamma order.

Solves with L inside inverse Lanczos are exact (sparse factorisation) by
default; inner="pcg" uses the paper's inner iteration (Sec. 4): PCG to a
relative residual inner_tol (1e-3 there) preconditioned by L restricted to
each face Gamma_i with the cross points removed (diagonal at cross points).
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import dd


class _Component:
    def __init__(self, pos, M, L, theta, groups=None, inner="exact", inner_tol=1e-3):
        self.pos = pos                      # positions in the Gamma vector
        self.M = sp.csc_matrix(M)
        self.L = sp.csc_matrix(L)
        self.theta = theta
        self.inner = inner
        self.inner_tol = inner_tol
        self.inner_its = []                 # inner PCG iterations per solve with L
        # face blocks of L (cross points removed) for the inner PCG
        Ld = self.L.toarray()
        self.groups = []
        self.cross = np.zeros(0, dtype=np.int64)
        if groups is not None:
            faces, cross = groups
            self.groups = [(g, np.linalg.inv(Ld[np.ix_(g, g)])) for g in faces]
            self.cross = np.asarray(cross, dtype=np.int64)
            self.cross_d = np.diag(Ld)[self.cross]
        mu, V = sla.eigh(L.toarray(), M.toarray())  # L V = M V diag(mu), V^T M V = I
        self.singular = mu[0] <= 1e-12 * max(mu[-1], 1.0)
        if self.singular:
            mu0 = np.where(mu <= 1e-12 * max(mu[-1], 1.0), 0.0, mu)
            lam = 1.0 + mu0 ** (1.0 - theta)
        else:
            lam = mu ** (1.0 - theta)
        self.V = V
        self.lam = lam
        self.Mlu = spla.splu(self.M)
        self.Llu = None if self.singular else spla.splu(self.L)

    def exact(self, r):
        return self.V @ ((self.V.T @ r) / self.lam)

    def _precond_L(self, r):
        z = np.zeros_like(r)
        for g, Linv in self.groups:
            z[g] = Linv @ r[g]
        z[self.cross] = r[self.cross] / self.cross_d
        return z

    def solve_L(self, b):
        """x = L^-1 b: exact, or the paper's inner PCG (Sec. 4)."""
        if self.inner == "exact":
            return self.Llu.solve(b)
        x = np.zeros_like(b)
        r = b.copy()
        z = self._precond_L(r)
        p = z.copy()
        rz = r @ z
        nb = np.linalg.norm(b)
        k = 0
        while np.linalg.norm(r) > self.inner_tol * nb and k < 1000:
            q = self.L @ p
            a = rz / (p @ q)
            x += a * p
            r -= a * q
            z = self._precond_L(r)
            rz_new = r @ z
            p = z + (rz_new / rz) * p
            rz = rz_new
            k += 1
        self.inner_its.append(k)
        return x

    def lanczos(self, r, k):
        """k steps of inverse Lanczos (full M-orthogonalisation)."""
        if self.singular:
            return self.exact(r)
        b = self.Mlu.solve(r)
        nb = np.sqrt(b @ (self.M @ b))
        if nb == 0.0:
            return np.zeros_like(r)
        n = len(r)
        k = min(k, n)
        Q = np.zeros((n, k + 1))
        alpha = np.zeros(k)
        beta = np.zeros(k)
        Q[:, 0] = b / nb
        m = k
        for j in range(k):
            w = self.solve_L(self.M @ Q[:, j])         # B q_j = L^-1 M q_j
            alpha[j] = Q[:, j] @ (self.M @ w)
            for i in range(j + 1):                      # M-orthogonalise against Q_j
                w = w - (Q[:, i] @ (self.M @ w)) * Q[:, i]
            beta[j] = np.sqrt(max(w @ (self.M @ w), 0.0))
            if j + 1 < k:
                if beta[j] <= 1e-14 * max(abs(alpha[: j + 1]).max(), 1e-300):
                    m = j + 1                            # invariant subspace: exact
                    break
                Q[:, j + 1] = w / beta[j]
        self.last_T = (alpha[:m].copy(), beta[: m - 1].copy())  # for step-by-step comparisons
        T = np.diag(alpha[:m]) + np.diag(beta[: m - 1], 1) + np.diag(beta[: m - 1], -1)
        t, U = np.linalg.eigh(T)
        f = np.clip(t, 0.0, None) ** (1.0 - self.theta)  # B^(1-theta), B SPD in <.,.>_M
        return nb * (Q[:, :m] @ (U @ (f * U[0, :])))


class GlobalPreconditioner:
    """z = S~^-1 r with S~ = Hhat_theta of eq. NumberNine on all of Gamma.

    steps: None for the exact application, else the number of inverse Lanczos
    steps.  face_scaling "dof" (reading Q8, default) scales every component by
    W = diag(sqrt(diag(K_GG) / diag(Htilde))) so that diag(S~) = diag(K_GG);
    "diag" (reading Q25) uses the surrogate diag(M)^theta diag(L)^(1-theta)
    in place of diag(Htilde), which needs no eigendecomposition of the whole
    interface (the form the GPU applies on large grids); False keeps the
    paper-literal Htilde (homogeneous problems only).
    """

    def __init__(self, dec, K, theta=0.5, steps=None, face_scaling="dof", inner="exact", inner_tol=1e-3):
        self.dec = dec
        self.steps = steps
        grid = dec.grid
        d = grid.dim
        G = dec.gamma_dofs
        M, L = dd.interface_mass_laplacian(dec)
        Kdiag = K.diagonal()
        self.comps = []
        for c in range(d):
            pos = np.array([k for k, g in enumerate(G) if int(g) % d == c], dtype=np.int64)
            if len(pos) == 0:
                continue
            nodes = np.array([int(G[k]) // d for k in pos])
            # faces (nodes of exactly two subdomains, grouped by the pair) and
            # cross points, as local indices of this component
            faces, cross = {}, []
            for i, n in enumerate(nodes):
                subs = dec.node_subs[n]
                if len(subs) == 2:
                    faces.setdefault(subs, []).append(i)
                else:
                    cross.append(i)
            groups = ([np.array(v) for _, v in sorted(faces.items(), key=lambda kv: sorted(kv[0]))], cross)
            comp = _Component(pos, M[nodes][:, nodes], L[nodes][:, nodes], theta, groups, inner, inner_tol)
            if face_scaling == "dof":
                Hdiag = np.einsum("ij,j,ij->i", comp.M.toarray() @ comp.V, comp.lam, comp.M.toarray() @ comp.V)
                comp.w = np.sqrt(Kdiag[G[pos]] / Hdiag)
            elif face_scaling == "diag":
                surrogate = comp.M.diagonal() ** theta * comp.L.diagonal() ** (1.0 - theta)
                comp.w = np.sqrt(Kdiag[G[pos]] / surrogate)
            else:
                comp.w = np.ones(len(pos))
            self.comps.append(comp)

    def apply(self, r):
        z = np.zeros_like(r)
        for c in self.comps:
            rc = r[c.pos] / c.w
            zc = c.exact(rc) if self.steps is None else c.lanczos(rc, self.steps)
            z[c.pos] = zc / c.w
        return z

    def dense(self):
        """S~^-1 (exact) as a dense matrix (small grids)."""
        n = len(self.dec.gamma_dofs)
        P = np.zeros((n, n))
        for c in self.comps:
            Wi = np.diag(1.0 / c.w)
            P[np.ix_(c.pos, c.pos)] = Wi @ (c.V @ np.diag(1.0 / c.lam) @ c.V.T) @ Wi
        return P
