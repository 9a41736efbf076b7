"""The seeded synthetic inputs match the recipes stated for them (CPU only):
GRF densities (reading Q19), the 64 uneven batched problems (Q20), the named
workloads' sizes and boundary conditions."""
import math

import numpy as np

import workloads


def test_grf_density_recipe():
    ne = (128, 64)
    a = workloads.grf_density(ne, 7)
    b = workloads.grf_density(ne, 7)
    c = workloads.grf_density(ne, 8)
    assert np.array_equal(a, b) and not np.array_equal(a, c)      # seeded
    assert a.shape == (128 * 64,) and a.min() >= 1e-3 and a.max() <= 1.0
    # the normal CDF of a standardised field: median near the middle of [1e-3, 1]
    assert abs(np.median(a) - (1e-3 + 0.5 * (1 - 1e-3))) < 0.1
    # smooth on the correlation length (sigma = 8 elements): neighbours in x
    # correlate strongly, elements 64 apart (periodic half-length) do not
    g = a.reshape(ne)
    z = g - g.mean()
    r1 = (z[1:, :] * z[:-1, :]).mean() / z.var()
    r64 = (z[64:, :] * z[:64, :]).mean() / z.var()
    assert r1 > 0.95 and abs(r64) < 0.3


def test_batch_problem_recipe():
    probs = workloads.batch_problems(base_seed=0, count=64)
    assert len(probs) == 64
    assert probs == workloads.batch_problems(base_seed=0, count=64)   # seeded
    subs = {p["sub"] for p in probs}
    assert subs == {8, 16, 32}
    for p in probs:
        nx, ny = p["ne"]
        s = p["sub"]
        assert ny * 2 == nx and nx % (2 * s) == 0 and nx >= 2 * s
        assert 64 - 2 * s <= nx <= 512 + 2 * s       # log-uniform target in [64, 512], rounded to 2s
        assert 0.2 <= p["nu"] <= 0.45 and p["p"] == 3.0 and p["E"] == 1.0
        assert p["density"][0] == "grf"
    # the targets are log-uniform: about half the grids below the geometric mean
    lo = sum(1 for p in probs if p["ne"][0] < math.sqrt(64 * 512))
    assert 16 <= lo <= 48


def test_named_workloads():
    c0, c1, c2, c4 = (workloads.config(n) for n in ("c0", "c1", "c2", "c4"))
    assert c0["ne"] == (64, 32) and c0["sub"] == 16 and c0["dim"] == 2
    assert c1["ne"] == (512, 256) and c1["sub"] == 16
    assert c2["ne"] == (96, 48, 48) and c2["sub"] == 8 and c2["dim"] == 3
    assert c4["ne"] == (256, 128) and c4["sub"] == 16 and c4["v_frac"] == 0.4
    rho1 = workloads.density(c1)
    assert rho1.shape == (512 * 256,) and 1e-3 <= rho1.min() and rho1.max() <= 1.0
    rho2 = workloads.density(c2)
    assert rho2.shape == (96 * 48 * 48,) and 1e-3 <= rho2.min() and rho2.max() <= 1.0
