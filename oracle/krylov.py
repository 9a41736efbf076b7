"""GMRES on the full block system (test infrastructure only).

Sec. 3: K P^-1 with P = [[K_II, K_IG], [0, S]] is block lower triangular with
identity diagonal blocks, so (K P^-1 - I)^2 = 0 and GMRES preconditioned from
the right with the exact P stops within two iterations (reading Q1 of the
printed minimal polynomial).  P~ replaces S by S~; P~^-1 is the three-factor
product written in Sec. 3.
"""
import numpy as np


def gmres(apply_A, b, tol=1e-10, max_it=200):
    """Unrestarted GMRES with modified Gram-Schmidt and Givens rotations.

    Returns (x, iterations, residual history).  Stops when the Arnoldi
    residual estimate drops to tol * ||b||.
    """
    n = len(b)
    beta = np.linalg.norm(b)
    V = np.zeros((max_it + 1, n))
    H = np.zeros((max_it + 1, max_it))
    cs = np.zeros(max_it)
    sn = np.zeros(max_it)
    e = np.zeros(max_it + 1)
    e[0] = beta
    V[0] = b / beta
    hist = [beta]
    k = 0
    for k in range(max_it):
        w = apply_A(V[k])
        for j in range(k + 1):
            H[j, k] = w @ V[j]
            w = w - H[j, k] * V[j]
        H[k + 1, k] = np.linalg.norm(w)
        if H[k + 1, k] > 0:
            V[k + 1] = w / H[k + 1, k]
        for j in range(k):
            t = cs[j] * H[j, k] + sn[j] * H[j + 1, k]
            H[j + 1, k] = -sn[j] * H[j, k] + cs[j] * H[j + 1, k]
            H[j, k] = t
        den = np.hypot(H[k, k], H[k + 1, k])
        cs[k] = H[k, k] / den
        sn[k] = H[k + 1, k] / den
        H[k, k] = den
        H[k + 1, k] = 0.0
        e[k + 1] = -sn[k] * e[k]
        e[k] = cs[k] * e[k]
        hist.append(abs(e[k + 1]))
        if hist[-1] <= tol * beta:
            k += 1
            break
    else:
        k = max_it
    y = np.linalg.solve(np.triu(H[:k, :k]), e[:k])
    x = V[:k].T @ y
    return x, k, hist


def block_right_preconditioner(dd, apply_Sinv):
    """v -> P~^-1 v for P~ = [[K_II, K_IG], [0, S~]] on the (I, G) ordering.

    P~^-1 = diag(K_II^-1, I) [[I, -K_IG], [0, I]] diag(I, S~^-1) (Sec. 3).
    Vectors are ordered (all interior DOFs by subdomain, then Gamma DOFs).
    """
    nI = sum(len(b[0]) for b in dd.blocks)

    def apply(v):
        vI, vG = v[:nI], v[nI:]
        wG = apply_Sinv(vG)
        out = np.empty_like(v)
        off = 0
        for I, cf, KIG in dd.blocks:
            m = len(I)
            rhs = vI[off:off + m] - KIG @ wG
            from scipy.linalg import cho_solve
            out[off:off + m] = cho_solve(cf, rhs)
            off += m
        out[nI:] = wG
        return out

    return apply


def fgmres(apply_A, apply_P, b, tol=1e-10, max_it=200):
    """Flexible GMRES (Saad 1993), right preconditioned: the preconditioned
    directions z_j = P_j^-1 v_j are kept, so P may change from step to step
    (Sec. 3: the inverse Lanczos application of S~^-1 depends on its input).
    Returns (x, iterations, residual history); x = Z_k y.
    """
    n = len(b)
    beta = np.linalg.norm(b)
    V = np.zeros((max_it + 1, n))
    Z = np.zeros((max_it, n))
    H = np.zeros((max_it + 1, max_it))
    cs = np.zeros(max_it)
    sn = np.zeros(max_it)
    e = np.zeros(max_it + 1)
    e[0] = beta
    V[0] = b / beta
    hist = [beta]
    k = 0
    for k in range(max_it):
        Z[k] = apply_P(V[k])
        w = apply_A(Z[k])
        for j in range(k + 1):
            H[j, k] = w @ V[j]
            w = w - H[j, k] * V[j]
        H[k + 1, k] = np.linalg.norm(w)
        if H[k + 1, k] > 0:
            V[k + 1] = w / H[k + 1, k]
        for j in range(k):
            t = cs[j] * H[j, k] + sn[j] * H[j + 1, k]
            H[j + 1, k] = -sn[j] * H[j, k] + cs[j] * H[j + 1, k]
            H[j, k] = t
        den = np.hypot(H[k, k], H[k + 1, k])
        cs[k] = H[k, k] / den
        sn[k] = H[k + 1, k] / den
        H[k, k] = den
        H[k + 1, k] = 0.0
        e[k + 1] = -sn[k] * e[k]
        e[k] = cs[k] * e[k]
        hist.append(abs(e[k + 1]))
        if hist[-1] <= tol * beta:
            k += 1
            break
    else:
        k = max_it
    y = np.linalg.solve(np.triu(H[:k, :k]), e[:k])
    x = Z[:k].T @ y
    return x, k, hist
