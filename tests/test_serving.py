"""Continuous-batching server: requests of different materials, sizes and horizons
submitted while others run give the same results as when run alone; admission follows the
memory budget; polling is non-blocking; served results match the FP64 oracle."""
import time

import numpy as np
import pytest

from oracle import fem
from oracle import oracle as orc
from paper_2412_12089_gb300 import mpm
from paper_2412_12089_gb300 import workloads as wl

from gpu_helpers import rel_err

pytestmark = pytest.mark.gpu


def mixed_requests(seed=0):
    rng = np.random.default_rng(seed)
    reqs = []
    d = wl.dough(n_envs=2, seed=seed, n_range=(800, 3000), substeps=6, T=5)
    f = wl.fluid(n_envs=2, seed=seed + 1, n=1500, substeps=5, T=4)
    j = wl.jumper(n_envs=1, seed=seed + 2, n=2500, G=48, substeps=4, T=3)
    sj = wl.softjumper(n_envs=1, seed=seed + 3, T=3)  # tetrahedral FEM
    for w in (d, f, j, sj):
        for e in range(w.n_envs):
            T = int(rng.integers(2, w.T + 1))
            A = w.specs[e].action_dim
            reqs.append((w.specs[e], w.inits[e], w.actions[:T, e, :max(A, 1)][:, :A], T, bool(rng.integers(0, 2))))
    return reqs


def run_alone(req):
    spec, init, acts, T, grad = req
    srv = mpm.mpm_server_create(mem_fraction=0.5, max_resident=4)
    try:
        t = mpm.mpm_submit(srv, spec, init, acts if acts.size else None, T, want_grad=grad)
        return mpm.mpm_wait(srv, t, 120000.0)
    finally:
        mpm.mpm_server_destroy(srv)


def test_mixed_stream_equals_alone():
    reqs = mixed_requests(3)
    srv = mpm.mpm_server_create(mem_fraction=0.5, max_resident=3)
    try:
        tickets = []
        for i, (spec, init, acts, T, grad) in enumerate(reqs):
            tickets.append(mpm.mpm_submit(srv, spec, init, acts if acts.size else None, T, want_grad=grad))
            if i % 2 == 1:
                time.sleep(0.05)  # later requests arrive while earlier ones run
        results = [mpm.mpm_wait(srv, t, 120000.0) for t in tickets]
        for t in tickets:
            mpm.mpm_release(srv, t)
    finally:
        mpm.mpm_server_destroy(srv)
    overlapped = 0
    for i, (req, res) in enumerate(zip(reqs, results)):
        assert res["status"] == 0, (i, res["status"])
        alone = run_alone(req)
        assert rel_err(res["x_final"], alone["x_final"]) < 1e-5, i
        assert np.allclose(res["rewards"], alone["rewards"], rtol=1e-5, atol=1e-7), i
        if req[4] and req[0].action_dim:
            assert rel_err(res["action_grad"], alone["action_grad"]) < 1e-4, i
        if req[0].material == "fem":  # FEM sums run in a fixed order: bitwise reproducible
            assert np.array_equal(res["x_final"], alone["x_final"]), i
            assert np.array_equal(res["rewards"], alone["rewards"]), i
        # at most max_resident requests resident at once; some overlapped in time
        others = [r for r in results if r is not res]
        if any(o["admit_ms"] < res["finish_ms"] and res["admit_ms"] < o["finish_ms"] for o in others):
            overlapped += 1
    assert overlapped >= 2
    events = sorted([(r["admit_ms"], 1) for r in results] + [(r["finish_ms"], -1) for r in results])
    live = peak = 0
    for _, d in events:
        live += d
        peak = max(peak, live)
    assert peak <= 3


def test_served_rollout_matches_oracle():
    w = wl.fluid(n_envs=1, seed=9, n=1200, substeps=4, T=3)
    s, init = w.specs[0], w.inits[0]
    acts = w.actions[:3, 0, :3]
    srv = mpm.mpm_server_create(mem_fraction=0.3, max_resident=2)
    try:
        t = mpm.mpm_submit(srv, s, init, acts, 3, want_grad=True, reward_adj=np.ones(3, np.float32))
        res = mpm.mpm_wait(srv, t, 120000.0)
    finally:
        mpm.mpm_server_destroy(srv)
    sp = orc.make_spec(s)
    st = orc.State.from_init(init)
    out, q, rew, _ = orc.rollout(sp, st, np.array(s.pose0, np.float64), acts.astype(np.float64))
    assert rel_err(res["x_final"], out.x) < 1e-3
    assert np.allclose(res["rewards"], rew, rtol=1e-3, atol=1e-6)
    ag, _, _ = orc.rollout_adj(sp, st, np.array(s.pose0, np.float64), acts.astype(np.float64), rbar=np.ones(3))
    assert rel_err(res["action_grad"], ag) < 1e-3


def test_poll_not_ready_then_ok_and_budget():
    w = wl.jumper(n_envs=1, seed=4, n=20000, G=64, substeps=10, T=6)
    s, init = w.specs[0], w.inits[0]
    acts = w.actions[:6, 0, :s.action_dim]
    srv = mpm.mpm_server_create(mem_fraction=0.5, max_resident=2)
    try:
        t = mpm.mpm_submit(srv, s, init, acts, 6, want_grad=True)
        assert mpm.mpm_poll(srv, t) is None
        res = mpm.mpm_wait(srv, t, 120000.0)
        assert res["status"] == 0 and mpm.mpm_poll(srv, t) is not None
    finally:
        mpm.mpm_server_destroy(srv)
    tiny = mpm.mpm_server_create(mem_fraction=1e-6, max_resident=2)
    try:
        with pytest.raises(mpm.MpmError) as ei:
            mpm.mpm_submit(tiny, s, init, acts, 6)
        assert ei.value.code == 8  # BUDGET
    finally:
        mpm.mpm_server_destroy(tiny)


def test_served_fem_rollout_matches_oracle():
    w = wl.softjumper(n_envs=1, seed=19, T=2)
    s, init = w.specs[0], w.inits[0]
    acts = w.actions[:2, 0, :s.n_groups]
    srv = mpm.mpm_server_create(mem_fraction=0.3, max_resident=2)
    try:
        t = mpm.mpm_submit(srv, s, init, acts, 2, want_grad=True, reward_adj=np.ones(2, np.float32))
        res = mpm.mpm_wait(srv, t, 120000.0)
    finally:
        mpm.mpm_server_destroy(srv)
    assert res["status"] == 0
    m = fem.make_mesh(s)
    x, v, r, _ = fem.rollout(m, init.x, init.v, acts)
    assert rel_err(res["x_final"], x) < 1e-3
    assert np.allclose(res["rewards"], r, rtol=1e-3, atol=1e-5)
    ag, _, _, _ = fem.rollout_adj(m, init.x, init.v, acts, rbar=np.ones(2))
    assert rel_err(res["action_grad"], ag) < 1e-3
