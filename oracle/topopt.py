"""Topology-optimisation step of Sec. 5 (test infrastructure only).

The problem is eq. NumberTen (min f^T u s.t. K(rho) u = f, volume bound,
density bounds) with element stiffness E rho_e^p K_e (p = 1 is the paper's
variable-thickness sheet; the workloads use SIMP p = 3, reading Q3).  The
Picard loop of Sec. 5 is: (1) finite-element analysis, (2) density update by
optimality criteria (OC), (3) convergence check.  The paper cites Bendsoe for
OC and gives no formula; the readings (Q15) are written here from the
mathematics of the Lagrangian stationarity condition:

* linear "hat" density filter rho~ = Hbar rho, Hbar_ij = w_ij / sum_k w_ik,
  w_ij = max(0, r_min - |c_i - c_j|) over element centres;
* compliance c = f^T u; dc/drho~_e = -p rho~_e^(p-1) E u_e^T K_e u_e
  (adjoint of the self-adjoint compliance); chain rule dc/drho = Hbar^T dc/drho~;
* volume V(rho~) = sum rho~ = (Hbar^T 1) . rho, so dV/drho = Hbar^T 1;
* OC fixed point rho_new = clamp(rho (-dc / (lambda dV))^(1/2),
  max(rho_min, rho - m), min(1, rho + m)) with move m = 0.2, the multiplier
  lambda found by 64 bisection steps on [0, 1e9] so that
  V(rho~_new) = v_frac * n_elem.

Sec. 5 (Table 3) solves each Picard step's linear system to an adaptive
tolerance "based on successive compliance values" and gives no formula; the
reading (Q23) is `adaptive_tolerance` below.
"""
import numpy as np
import scipy.sparse as sp


def filter_matrix(ne, r_min):
    """Row-normalised hat-filter matrix Hbar on the element grid (2D or 3D)."""
    dim = len(ne)
    R = int(np.ceil(r_min)) - 1 if float(r_min).is_integer() else int(np.floor(r_min))
    axes = [np.arange(n) for n in ne]
    centres = np.stack([m.ravel() for m in np.meshgrid(*axes, indexing="ij")], axis=1)
    n = len(centres)

    def eidx(c):
        idx = np.zeros(len(c), dtype=np.int64)
        for a in range(dim):
            idx = idx * ne[a] + c[:, a]
        return idx

    rows, cols, vals = [], [], []
    offsets = np.stack([m.ravel() for m in np.meshgrid(*([np.arange(-R, R + 1)] * dim),
                                                       indexing="ij")], axis=1)
    for off in offsets:
        dist = np.sqrt(np.sum(off.astype(float) ** 2))
        w = r_min - dist
        if w <= 0:
            continue
        nb = centres + off
        ok = np.all((nb >= 0) & (nb < np.array(ne)), axis=1)
        rows.append(np.nonzero(ok)[0])
        cols.append(eidx(nb[ok]))
        vals.append(np.full(ok.sum(), w))
    W = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    s = np.asarray(W.sum(axis=1)).ravel()
    return sp.diags(1.0 / s) @ W


def compliance_and_sensitivity(grid, Ke, E, p, rho_f, u, f):
    """c = f^T u and dc/drho~ for element densities rho_f (physical)."""
    edofs = grid.element_dofs()
    ue = u[edofs]
    energy = np.einsum("ei,ij,ej->e", ue, Ke, ue)
    c = float(f @ u)
    dc = -p * E * rho_f ** (p - 1) * energy
    return c, dc


def oc_update(rho, dc, dv, v_target, rho_min=1e-3, move=0.2, steps=64, lam_hi=1e9):
    """Optimality-criteria update with bisection on the volume multiplier."""
    lo, hi = 0.0, lam_hi
    B = np.maximum(-dc, 0.0) / dv
    lower = np.maximum(rho_min, rho - move)
    upper = np.minimum(1.0, rho + move)
    new = rho
    for _ in range(steps):
        lam = 0.5 * (lo + hi)
        new = np.clip(rho * np.sqrt(B / lam), lower, upper) if lam > 0 else upper
        if dv @ new > v_target:
            lo = lam
        else:
            hi = lam
    lam = 0.5 * (lo + hi)
    new = np.clip(rho * np.sqrt(B / lam), lower, upper)
    return new, lam


def topopt_step(grid, Ke, E, p, Hbar, rho, f, solve, v_frac, rho_min=1e-3, move=0.2):
    """One Picard step of Sec. 5: filter, FEA solve, sensitivities, OC.

    `solve(factors) -> u` performs the finite-element analysis for element
    stiffness factors E rho~^p.  Returns (rho_new, compliance, u, rho~).
    """
    rho_f = Hbar @ rho
    u = solve(E * rho_f ** p)
    c, dcf = compliance_and_sensitivity(grid, Ke, E, p, rho_f, u, f)
    dc = Hbar.T @ dcf
    dv = Hbar.T @ np.ones(len(rho))
    new, _ = oc_update(rho, dc, dv, v_frac * len(rho), rho_min, move)
    return new, c, u, rho_f


def adaptive_tolerance(history, eta, tol_min, tol_max):
    """Krylov tolerance of the next Picard step from the compliances of the
    steps so far (Sec. 5, Table 3; reading Q23): the relative change of the
    last two compliances, scaled by eta, clamped to [tol_min, tol_max]; tol_max
    while fewer than two compliances are known.  A step whose design still
    moves the compliance by a relative d needs its analysis no more accurate
    than a fraction eta of d."""
    tol_max = max(tol_max, tol_min)
    if len(history) < 2:
        return tol_max
    c1, c0 = history[-1], history[-2]
    return min(tol_max, max(tol_min, eta * abs(c1 - c0) / abs(c1)))
