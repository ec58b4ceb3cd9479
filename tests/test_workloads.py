"""The synthetic workloads carry the paper's printed task constants (App. E tables,
stored in tests/golden/task_constants.txt) and are deterministic in their seed."""
import os

import numpy as np

from paper_2412_12089_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "task_constants.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        task, key, val = line.split()[:3]
        out[(task, key)] = float(np.float32(val))  # spec inputs are FP32-representable
    return out


def test_dough_matches_rollingflat_table():
    g = golden()
    w = wl.dough(n_envs=3, seed=1, T=2)
    for s in w.specs:
        assert s.grid_res == g[("RollingFlat", "N_g")]
        assert s.dt == g[("RollingFlat", "dt")]
        assert s.rho == g[("RollingFlat", "rho")] and s.E == g[("RollingFlat", "E")]
        assert s.nu == g[("RollingFlat", "nu")] and s.yield_stress == g[("RollingFlat", "sigma_y")]
        assert s.coll_mu == g[("RollingFlat", "mu_b")] and s.rparam[0] == g[("RollingFlat", "h_flat")]
        assert s.n_sub == g[("RollingFlat", "obs_particles")]
        assert 2000 <= s.n_particles <= 16000


def test_fluid_and_jumper_match_tables():
    g = golden()
    f = wl.fluid(n_envs=2, seed=1, n=512, T=2)
    for s in f.specs:
        assert s.dt == g[("FluidMove", "dt")] and s.rho == g[("FluidMove", "rho")]
        assert s.coll_mu == g[("FluidMove", "mu_b")] and s.n_sub == g[("FluidMove", "obs_particles")]
    j = wl.jumper(n_envs=1, seed=1, n=2000, G=32, T=2)
    s = j.specs[0]
    assert s.n_groups == g[("SoftJumper", "actions")]
    assert s.rparam[1] == g[("SoftJumper", "k_up")] and s.rparam[2] == g[("SoftJumper", "k_a")]
    grp = j.inits[0].group
    assert grp.max() < s.n_groups and (grp >= 0).any() and (grp < 0).any()


def test_seeded_and_fp32():
    a = wl.dough(n_envs=2, seed=5, T=3)
    b = wl.dough(n_envs=2, seed=5, T=3)
    for ia, ib in zip(a.inits, b.inits):
        assert ia.x.dtype == np.float32 and np.array_equal(ia.x, ib.x)
    assert np.array_equal(a.actions, b.actions)
    c = wl.cube(seed=0)
    x = c.inits[0].x
    assert x.shape == (4096, 3) and x.min() >= 0.4 and x.max() <= 0.6
