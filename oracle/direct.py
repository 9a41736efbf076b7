"""Global sparse direct solve of K u = f (test infrastructure only).

The DD method of Sec. 2 (eq. 3MatSplit2) reaches the exact solution of
K(rho) u = f up to rounding, so the oracle for the final displacement is that
definition: SuperLU on the free-DOF system plus FP64 iterative refinement with
the residual accumulated in extended precision where the platform has it.
"""
import numpy as np
import scipy.sparse.linalg as spla


def solve(K, f, fixed, refine=2):
    """u with K_ff u_f = f_f, u = 0 on fixed DOFs.  K is the full (n_dof) matrix."""
    free = np.nonzero(~np.asarray(fixed, dtype=bool))[0]
    Kff = K[free][:, free].tocsc()
    lu = spla.splu(Kff)
    ff = f[free]
    uf = lu.solve(ff)
    Kl = Kff.astype(np.longdouble) if np.finfo(np.longdouble).eps < np.finfo(float).eps else None
    for _ in range(refine):
        if Kl is not None:
            r = (ff.astype(np.longdouble) - Kl @ uf.astype(np.longdouble)).astype(float)
        else:
            r = ff - Kff @ uf
        uf = uf + lu.solve(r)
    u = np.zeros(K.shape[0])
    u[free] = uf
    return u


def rel_residual(K, f, u, fixed):
    free = ~np.asarray(fixed, dtype=bool)
    r = (f - K @ u)[free]
    return np.linalg.norm(r) / np.linalg.norm(f[free])
