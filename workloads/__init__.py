"""Seeded synthetic workloads (shared by the oracle, the tests and bench.py).

This module holds input generators and workload descriptions only: grid and
subdomain sizes, material constants, boundary-condition specifications and
seeded density fields.  It contains none of the method's arithmetic (no
stiffness, no decomposition, no solve) and imports neither the oracle nor the
GPU library.

Boundary-condition specs are plain dicts understood by both sides:
  "clamp":    list of (axis, side): every DOF on that grid face is fixed;
  "fix":      list of ((i, j[, k]), component): single fixed DOFs;
  "point":    list of ((i, j[, k]), force vector): nodal point loads;
  "traction": (axis, side, traction vector): uniform surface traction on a face.
"""
import math

import numpy as np
from scipy.special import ndtr


def cantilever_2d(nx, ny):
    """Left edge clamped, unit downward point load at the right mid-edge node."""
    return {"clamp": [(0, 0)], "point": [((nx, ny // 2), (0.0, -1.0))]}


def mbb_half_2d(nx, ny):
    """MBB half-beam: symmetry u_x = 0 on x = 0, roller u_y = 0 at the bottom-right
    node, unit downward load at the top-left node (reading Q17)."""
    fix = [((0, j), 0) for j in range(ny + 1)] + [((nx, 0), 1)]
    return {"fix": fix, "point": [((0, ny), (0.0, -1.0))]}


def cantilever_3d(nx, ny, nz):
    """Face x = 0 clamped; uniform traction of total force 1 in -z on face x = nx
    (reading Q18)."""
    return {"clamp": [(0, 0)], "traction": (0, 1, (0.0, 0.0, -1.0 / (ny * nz)))}


def table1_2d(h_inv):
    """Loads of the paper's Table 1 test problem on (0,2)x(0,1) (reading Q14)
    for a grid of unit elements standing for elements of width h = 1/h_inv:
    right edge clamped, downward body force 0.75 (0.75 h^2 per unit element)
    and outward unit traction on the left edge x = 0 (normal (-1, 0); h per
    unit edge)."""
    h = 1.0 / h_inv
    return {"clamp": [(0, 1)], "traction": (0, 0, (-h, 0.0)), "body": (0.0, -0.75 * h * h)}


def table1_config(h_inv, n_sub_x):
    """Table 1's cantilever on (0,2)x(0,1) with mesh width 1/h_inv: a
    (2 h_inv) x h_inv grid of unit elements (lengths in units of h) in
    n_sub_x x n_sub_x / 2 square subdomains; homogeneous material (rho = 1,
    p = 1), E = 1, nu = 0.3."""
    nx, ny = 2 * h_inv, h_inv
    sub = nx // n_sub_x
    return dict(name=f"table1_h{h_inv}_n{n_sub_x * n_sub_x // 2}", dim=2, ne=(nx, ny), sub=sub, E=1.0,
                nu=0.3, p=1.0, bc=table1_2d(h_inv), density=("uniform", 1.0))


def uniform_density(n_elem, value):
    return np.full(n_elem, float(value))


def grf_density(ne, seed, corr_len=8.0, rho_min=1e-3):
    """Gaussian-random-field densities in [rho_min, 1] (reading Q19).

    Standard normal noise on the element grid from numpy's default_rng(seed),
    periodic FFT smoothing with a Gaussian of standard deviation corr_len
    elements, standardised, then mapped through the normal CDF.  Flattened in
    element order (x-major).
    """
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(ne)
    fz = np.fft.fftn(z)
    k2 = np.zeros(ne)
    for a, n in enumerate(ne):
        f = np.fft.fftfreq(n)
        shape = [1] * len(ne)
        shape[a] = n
        k2 = k2 + (f ** 2).reshape(shape)
    z = np.real(np.fft.ifftn(fz * np.exp(-2.0 * math.pi ** 2 * corr_len ** 2 * k2)))
    z = (z - z.mean()) / z.std()
    return (rho_min + (1.0 - rho_min) * ndtr(z)).ravel()


def uniform_random_density(n_elem, seed, rho_min=1e-3):
    rng = np.random.default_rng(seed)
    return rng.uniform(rho_min, 1.0, n_elem)


def config(name):
    """Workload descriptions (sizes, material, BCs, density recipe)."""
    if name == "c0":
        nx, ny = 64, 32
        return dict(name=name, dim=2, ne=(nx, ny), sub=16, E=1.0, nu=0.3, p=3.0,
                    bc=cantilever_2d(nx, ny), density=("uniform", 0.5))
    if name == "c1":
        nx, ny = 512, 256
        return dict(name=name, dim=2, ne=(nx, ny), sub=16, E=1.0, nu=0.3, p=3.0,
                    bc=cantilever_2d(nx, ny), density=("grf", 0))
    if name == "c2":
        nx, ny, nz = 96, 48, 48
        return dict(name=name, dim=3, ne=(nx, ny, nz), sub=8, E=1.0, nu=0.3, p=3.0,
                    bc=cantilever_3d(nx, ny, nz), density=("uniform_random", 0))
    if name == "c4":
        nx, ny = 256, 128
        return dict(name=name, dim=2, ne=(nx, ny), sub=16, E=1.0, nu=0.3, p=3.0,
                    bc=mbb_half_2d(nx, ny), density=("uniform", 0.4),
                    v_frac=0.4, r_min=1.5, steps=100)
    raise KeyError(name)


def small_config(nx, ny, sub, seed=None, bc="cantilever", nu=0.3, p=3.0, nz=None):
    """Reduced-size variant of the workloads for parity tests."""
    if nz is not None:
        return dict(name=f"3d_{nx}x{ny}x{nz}_s{sub}", dim=3, ne=(nx, ny, nz), sub=sub,
                    E=1.0, nu=nu, p=p, bc=cantilever_3d(nx, ny, nz),
                    density=("uniform_random", seed if seed is not None else 0))
    spec = cantilever_2d(nx, ny) if bc == "cantilever" else mbb_half_2d(nx, ny)
    dens = ("grf", seed) if seed is not None else ("uniform", 0.5)
    return dict(name=f"2d_{nx}x{ny}_s{sub}", dim=2, ne=(nx, ny), sub=sub, E=1.0, nu=nu,
                p=p, bc=spec, density=dens)


def density(cfg):
    kind = cfg["density"][0]
    n_elem = int(np.prod(cfg["ne"]))
    if kind == "uniform":
        return uniform_density(n_elem, cfg["density"][1])
    if kind == "grf":
        return grf_density(cfg["ne"], cfg["density"][1])
    if kind == "uniform_random":
        return uniform_random_density(n_elem, cfg["density"][1])
    raise KeyError(kind)


def batch_problems(base_seed=0, count=64):
    """Batched uneven 2D problems (reading Q20).

    s ~ U{8,16,32}; nx = 2 s round(exp(U[ln 64, ln 512]) / (2 s)) (at least 2 s),
    ny = nx / 2; nu ~ U[0.2, 0.45]; GRF densities with seed base_seed + k;
    cantilever boundary conditions.
    """
    out = []
    for k in range(count):
        rng = np.random.default_rng(base_seed + 1000003 * (k + 1))
        s = int(rng.choice([8, 16, 32]))
        target = math.exp(rng.uniform(math.log(64), math.log(512)))
        nx = max(2 * s, 2 * s * int(round(target / (2 * s))))
        ny = nx // 2
        nu = float(rng.uniform(0.2, 0.45))
        out.append(dict(name=f"batch{k}", dim=2, ne=(nx, ny), sub=s, E=1.0, nu=nu, p=3.0,
                        bc=cantilever_2d(nx, ny), density=("grf", base_seed + k)))
    return out
