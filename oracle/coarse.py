"""Coarse space for the interface PCG (test infrastructure only).

Not part of the paper's method, whose preconditioner is purely face-local
(Sec. 4, eq. NumberEight/NumberNine); this module states the additive coarse
correction and the Galerkin initial guess that the solver adds on top of it:

  Q      orthonormal basis of span(Z) (columns of Z that are numerically
         dependent are dropped),
  E      = Q^T S Q   (k x k, must be SPD, else the coarse space is unusable),
  x0     = Q E^-1 Q^T g   (the S-orthogonal projection of S^-1 g onto span(Q);
         discarded when ||g - S x0|| > ||g||),
  P_c r  = P r + Q E^-1 Q^T r   (additive, SPD when P and E are),
  P_d r  = Q E^-1 Q^T r + (I - Q E^-1 Q^T S) P r   (deflation, the "A-DEF2"
         form of Tang, Nabben, Vuik and Erlangga, J. Sci. Comput. 39 (2009):
         eigenvalue 1 on span(Q) and the preconditioned spectrum elsewhere).
"""
import numpy as np


def orthonormal_basis(Z, drop=1e-10):
    """Modified Gram-Schmidt on the columns of Z (n x k), in column order.

    A column whose remaining norm is below drop * (its original norm) is
    dropped.  Returns Q (n x k') with k' <= k.
    """
    cols = []
    for j in range(Z.shape[1]):
        v = Z[:, j].astype(float).copy()
        n0 = np.linalg.norm(v)
        if n0 == 0.0:
            continue
        for q in cols:
            v -= (q @ v) * q
        nv = np.linalg.norm(v)
        if nv > drop * n0:
            cols.append(v / nv)
    return np.stack(cols, axis=1) if cols else np.zeros((Z.shape[0], 0))


class CoarseSpace:
    def __init__(self, apply_S, Z, drop=1e-10):
        self.Q = orthonormal_basis(Z, drop)
        k = self.Q.shape[1]
        self.SQ = np.stack([apply_S(self.Q[:, i]) for i in range(k)], axis=1) if k else self.Q.copy()
        E = self.Q.T @ self.SQ
        self.E = 0.5 * (E + E.T)
        try:
            self.L = np.linalg.cholesky(self.E) if k else np.zeros((0, 0))
            self.spd = True
        except np.linalg.LinAlgError:
            self.L = None
            self.spd = False

    @property
    def k(self):
        return self.Q.shape[1]

    def solve_E(self, y):
        return np.linalg.solve(self.L.T, np.linalg.solve(self.L, y))

    def x0(self, g):
        """Galerkin initial guess, or None when it does not reduce ||r||."""
        if not self.spd or self.k == 0:
            return None
        c = self.solve_E(self.Q.T @ g)
        x0 = self.Q @ c
        if np.linalg.norm(g - self.SQ @ c) > np.linalg.norm(g):
            return None
        return x0

    def preconditioner(self, apply_P):
        if not self.spd or self.k == 0:
            return apply_P
        return lambda r: apply_P(r) + self.Q @ self.solve_E(self.Q.T @ r)

    def deflated_preconditioner(self, apply_P):
        if not self.spd or self.k == 0:
            return apply_P

        def apply(r):
            z = apply_P(r)
            # Q^T S z = (S Q)^T z, S symmetric
            return z + self.Q @ self.solve_E(self.Q.T @ r - self.SQ.T @ z)
        return apply


def coarse_pcg(apply_S, apply_P, g, Z, tol, max_it, ref_norm=None, deflate=False):
    """Interface PCG with the coarse space of Z: Galerkin x0 and the additive
    (or, with deflate, the deflation) correction.  Returns (x, iterations,
    history, coarse_space)."""
    from oracle.dd import pcg
    cs = CoarseSpace(apply_S, Z)
    x0 = cs.x0(g)
    ref = np.linalg.norm(g) if ref_norm is None else ref_norm
    P = cs.deflated_preconditioner(apply_P) if deflate else cs.preconditioner(apply_P)
    x, it, hist = pcg(apply_S, P, g, tol, max_it, x0=x0, ref_norm=ref)
    return x, it, hist, cs
