"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (infinity-norm relative errors, per environment and quantity):
  one substep from the same FP32 state .......... 1e-5 on x, v, F (C: 1e-4)
  a control-step horizon ......................... 1e-3
  gradients against the FP64 oracle .............. 1e-3
  binning ........................................ bit-exact
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2412_12089_gb300 import workloads as wl

from gpu_helpers import gpu_run, oracle_run, perturb, rel_err, split

pytestmark = pytest.mark.gpu


def small(name, seed=0, substeps=None, T=1, **kw):
    if name == "cube":
        w = wl.cube(seed=seed, n=kw.pop("n", 1000), G=kw.pop("G", 32), substeps=substeps or 1, T=T)
    elif name == "dough":
        w = wl.dough(n_envs=kw.pop("n_envs", 3), seed=seed, n_range=kw.pop("n_range", (500, 3000)),
                     substeps=substeps or 1, T=T)
    elif name == "fluid":
        w = wl.fluid(n_envs=kw.pop("n_envs", 2), seed=seed, n=kw.pop("n", 1500), substeps=substeps or 1, T=T)
    elif name == "handflip":
        w = wl.handflip(n_envs=kw.pop("n_envs", 2), seed=seed, n=kw.pop("n", 1500), substeps=substeps or 1, T=T,
                        n_caps=kw.pop("n_caps", 6))
    elif name == "jumper":
        w = wl.jumper(n_envs=kw.pop("n_envs", 2), seed=seed, n=kw.pop("n", 3000), G=kw.pop("G", 48),
                      substeps=substeps or 1, T=T)
    else:
        raise ValueError(name)
    return w


# ------------------------------------------------------------------ binning

@pytest.mark.parametrize("n,G", [(1, 32), (1000, 32), (100_003, 48), (300_000, 96)])
def test_bin_bitexact(n, G):
    import torch

    from paper_2412_12089_gb300 import mpm

    rng = np.random.default_rng(n)
    x = (0.05 + 0.9 * rng.random((n, 3))).astype(np.float32)
    k = min(n, 500)
    x[:k] = ((np.floor(x[:k] * G - 0.5) + 0.5) / G).astype(np.float32)  # on cell boundaries
    xd = torch.as_tensor(x).cuda()
    keys = torch.empty(n, dtype=torch.int32, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    mpm.mpm_bin(xd, n, G, keys, perm)
    torch.cuda.synchronize()
    kg = keys.cpu().numpy().view(np.uint32)
    pg = perm.cpu().numpy().view(np.uint32)
    ko = orc.bin_keys_f32(x, G)
    assert np.array_equal(kg, ko)
    assert np.array_equal(pg, orc.stable_sort(ko))


# ------------------------------------------------------------------ one substep

@pytest.mark.parametrize("name", ["cube", "dough", "fluid", "jumper", "handflip"])
def test_substep_parity(name):
    w = perturb(small(name, seed=1, substeps=1, T=1), seed=2)
    b, rew, st = gpu_run(w, 1)
    for e in range(w.n_envs):
        o, q, r = oracle_run(w, e, 1)
        xs = split(w, st["x"])[e]
        vs = split(w, st["v"])[e]
        Cs = split(w, st["C"])[e]
        Fs = split(w, st["F"])[e]
        assert rel_err(xs, o.x) < 1e-5, (name, e, "x", rel_err(xs, o.x))
        assert rel_err(vs, o.v) < 1e-5, (name, e, "v", rel_err(vs, o.v))
        assert rel_err(Fs, o.F) < 1e-5, (name, e, "F", rel_err(Fs, o.F))
        assert rel_err(Cs, o.C) < 1e-4, (name, e, "C", rel_err(Cs, o.C))
        assert np.allclose(st["pose"][e], q[:4], atol=1e-6)  # body 0
        if w.specs[e].reward != "none":
            assert abs(rew[0, e] - r[0]) <= 1e-4 * max(1.0, abs(r[0])), (name, e, rew[0, e], r[0])
    code, flags = b.check_status()
    assert code == 0 and not flags.any()


@pytest.mark.parametrize("name", ["cube", "fluid", "jumper", "handflip"])
def test_substep_parity_warp_scatter(name, monkeypatch):
    """One substep and its gradient with the one-warp scatter shape (64-particle CTAs), for
    the materials and colliders the dough case of test_scatter_box_builds_match_oracle does
    not cover."""
    monkeypatch.setenv("MPM_SCATTER_BOX", "256")
    w = perturb(small(name, seed=1, substeps=1, T=1), seed=2)
    b, rew, st = gpu_run(w, 1)
    for e in range(w.n_envs):
        o, q, r = oracle_run(w, e, 1)
        for k, tol in (("x", 1e-5), ("v", 1e-5), ("F", 1e-5), ("C", 1e-4)):
            got = split(w, st[k])[e]
            assert rel_err(got, getattr(o, k)) < tol, (name, e, k, rel_err(got, getattr(o, k)))
    b.close()
    g, _ = _gpu_grads(w, 1, xbT=lambda x: 2.0 * x, rbar=np.ones((1, w.n_envs), np.float32))
    for e in range(w.n_envs):
        s = w.specs[e]
        sp = orc.make_spec(s)
        so = orc.State.from_init(w.inits[e])
        A = s.action_dim
        acts = w.actions[:1, e, :max(A, 1)].astype(np.float64)
        out, _, _, _ = orc.rollout(sp, so, orc.initial_pose(s), acts)
        ag, (xb, vb, Cb, Fb), _ = orc.rollout_adj(sp, so, orc.initial_pose(s), acts,
                                                  adj_final=(2.0 * out.x, None, None, None), rbar=np.ones(1))
        assert rel_err(split(w, g["xb0"])[e], xb) < 1e-3, (name, e)
        assert rel_err(split(w, g["vb0"])[e], vb) < 1e-3, (name, e)
        if A:
            assert rel_err(g["action_grad"][:, e, :A], ag) < 1e-3, (name, e)


# ------------------------------------------------------------------ horizons

def test_cube_horizon_c1():
    """The single-environment neo-Hookean cube at its full size: 4096 particles, 32^3 grid,
    50 substeps."""
    w = wl.cube(seed=0)
    w.specs[0] = w.specs[0].replace(substeps=50)
    b, rew, st = gpu_run(w, 1)
    o, q, r = oracle_run(w, 0, 1)
    for k in ("x", "v", "F"):
        assert rel_err(st[k], getattr(o, k)) < 1e-3, (k, rel_err(st[k], getattr(o, k)))


@pytest.mark.parametrize("name,T,S", [("dough", 2, 20), ("fluid", 2, 25), ("jumper", 2, 20), ("handflip", 2, 40)])
def test_horizon_parity(name, T, S):
    w = small(name, seed=3, substeps=S, T=T)
    b, rew, st = gpu_run(w, T)
    for e in range(w.n_envs):
        o, q, r = oracle_run(w, e, T)
        for k in ("x", "v", "F"):
            got = split(w, st[k])[e]
            assert rel_err(got, getattr(o, k)) < 1e-3, (name, e, k, rel_err(got, getattr(o, k)))
        assert np.allclose(rew[:, e], r, rtol=1e-3, atol=1e-5), (name, e, rew[:, e], r)


def test_container_floor_on_node_lattice():
    """The fluid container with its floor's top face exactly on a plane of grid nodes (and no
    vertical actions, so it stays there): nodes with zero signed distance take the full
    contact projection on both sides.  One substep at 1e-5 and a two-control-step horizon and
    its action gradients at 1e-3 against the oracle."""
    w = wl.fluid(n_envs=2, seed=23, n=1500, substeps=1, T=1, floor_cells=2.0, az=6 / 64)
    w.actions[:, :, 2] = 0.0
    for e, s in enumerate(w.specs):  # the floor's top face: a whole number of cells
        zf = (np.float32(s.pose0[2]) - np.float32(s.coll_dims[2])) * np.float32(s.grid_res)
        assert zf == 7.0, zf
    w = perturb(w, seed=4, v_std=0.5)
    for i in w.inits:  # particles moving down onto the floor
        i.v[:, 2] = -np.abs(i.v[:, 2])
    b, rew, st = gpu_run(w, 1)
    for e in range(w.n_envs):
        o, q, r = oracle_run(w, e, 1)
        for k, tol in (("x", 1e-5), ("v", 1e-5), ("F", 1e-5)):
            assert rel_err(split(w, st[k])[e], getattr(o, k)) < tol, (e, k, rel_err(split(w, st[k])[e], getattr(o, k)))
    b.close()
    T = 2
    w2 = wl.fluid(n_envs=2, seed=23, n=1500, substeps=25, T=T, floor_cells=2.0, az=6 / 64)
    w2.actions[:, :, 2] = 0.0
    g, st2 = _gpu_grads(w2, T, rbar=np.ones((T, 2), np.float32))
    for e in range(2):
        s = w2.specs[e]
        sp = orc.make_spec(s)
        so = orc.State.from_init(w2.inits[e])
        acts = w2.actions[:T, e, :3].astype(np.float64)
        o, _, _, _ = orc.rollout(sp, so, orc.initial_pose(s), acts)
        assert rel_err(split(w2, st2["x"].cpu().numpy())[e], o.x) < 1e-3
        ag, _, _ = orc.rollout_adj(sp, so, orc.initial_pose(s), acts, rbar=np.ones(T))
        assert rel_err(g["action_grad"][:, e, :3], ag) < 1e-3, (e, rel_err(g["action_grad"][:, e, :3], ag))


# ------------------------------------------------------------------ batching

def test_batched_equals_alone_and_per_env_launch():
    """Uneven environments stepped together give each environment's own result, and the
    one-launch-per-environment path gives the same result as the batched one."""
    w = small("dough", seed=5, substeps=4, T=2, n_envs=4, n_range=(200, 5000))
    _, rew_b, st_b = gpu_run(w, 2)
    _, rew_p, st_p = gpu_run(w, 2, per_env=True)
    assert rel_err(st_p["x"], st_b["x"]) < 1e-6
    assert np.allclose(rew_p, rew_b, rtol=1e-5, atol=1e-7)
    for e in range(w.n_envs):
        we = wl.Workload("one", [w.specs[e]], [w.inits[e]], w.actions[:, e:e + 1, :], w.T)
        _, rew_1, st_1 = gpu_run(we, 2)
        assert rel_err(st_1["x"], split(w, st_b["x"])[e]) < 1e-6
        assert np.allclose(rew_1[:, 0], rew_b[:, e], rtol=1e-5, atol=1e-7)


def test_graphs_equal_direct_launches():
    w = small("fluid", seed=6, substeps=5, T=3)
    _, rew_g, st_g = gpu_run(w, 3, use_graphs=True)
    _, rew_d, st_d = gpu_run(w, 3, use_graphs=False)
    assert rel_err(st_g["x"], st_d["x"]) < 1e-6
    assert np.allclose(rew_g, rew_d, rtol=1e-5, atol=1e-7)


def test_edge_cases_tiny_envs():
    """Single-particle and sub-warp environments next to a normal one."""
    w = small("cube", seed=7, substeps=3, T=1, n=700)
    s0, i0 = w.specs[0], w.inits[0]
    specs = [s0.replace(n_particles=1, p_vol=s0.p_vol), s0.replace(n_particles=17), s0]
    inits = [wl.EnvInit(i0.x[:1].copy(), i0.v[:1].copy(), i0.C[:1].copy(), i0.F[:1].copy()),
             wl.EnvInit(i0.x[:17].copy(), i0.v[:17].copy(), i0.C[:17].copy(), i0.F[:17].copy()), i0]
    w2 = wl.Workload("tiny", specs, inits, np.zeros((1, 3, 1), np.float32), 1)
    _, _, st = gpu_run(w2, 1)
    for e in range(3):
        o, _, _ = oracle_run(w2, e, 1)
        assert rel_err(split(w2, st["x"])[e], o.x) < 1e-5


def test_edge_cases_tiny_envs_gradients():
    """The reverse pass of single-particle and sub-warp environments next to a normal one:
    gradients of a random linear loss on the final positions, two recorded control steps."""
    T = 2
    w = small("cube", seed=17, substeps=3, T=T, n=700)
    s0, i0 = w.specs[0], w.inits[0]
    specs = [s0.replace(n_particles=1), s0.replace(n_particles=17), s0]
    inits = [wl.EnvInit(i0.x[:k].copy(), i0.v[:k].copy(), i0.C[:k].copy(), i0.F[:k].copy()) for k in (1, 17)] + [i0]
    w2 = wl.Workload("tiny", specs, inits, np.zeros((T, 3, 1), np.float32), T)
    xw = np.random.default_rng(18).standard_normal((w2.n_particles, 3)).astype(np.float32)
    g, _ = _gpu_grads(w2, T, xbT=lambda xT: xw)
    for e in range(3):
        sp = orc.make_spec(specs[e])
        so = orc.State.from_init(inits[e])
        _, (xb, vb, Cb, Fb), _ = orc.rollout_adj(sp, so, np.zeros(4), np.zeros((T, 1)),
                                                 adj_final=(split(w2, xw)[e].astype(np.float64), None, None, None))
        # a lone particle's stress momentum cancels exactly in G2P (v_p = v), so its F gradient
        # is zero up to rounding and has no relative error to compare
        quantities = (("x", g["xb0"], xb), ("v", g["vb0"], vb)) + ((("F", g["Fb0"], Fb),) if e else ())
        for name, gg, ref in quantities:
            assert rel_err(split(w2, gg)[e], ref) < 1e-3, (e, name, rel_err(split(w2, gg)[e], ref))


def test_maximum_env_size_and_grid():
    """The largest environment the ABI takes: 1,048,575 particles (the 20-bit particle id) on
    the largest grid, 128^3, one substep from a perturbed state, against the oracle; about
    60 particles per cell, so the scatter's cell groups are far larger than in the tasks."""
    w = perturb(wl.cube(seed=11, n=(1 << 20) - 1, G=128, substeps=1, T=1), seed=12)
    b, _, st = gpu_run(w, 1)
    try:
        code, flags = b.check_status()
    finally:
        b.close()
    assert code == 0 and not flags.any()
    o, _, _ = oracle_run(w, 0, 1)
    for k in ("x", "v", "F"):
        assert rel_err(st[k], getattr(o, k)) < 1e-5, (k, rel_err(st[k], getattr(o, k)))


def test_domain_status_flag():
    w = small("cube", seed=8, substeps=1, T=1, n=300)
    w.inits[0].x[5] = np.array([0.001, 0.5, 0.5], np.float32)  # below the first cell: base clamped
    b, _, _ = gpu_run(w, 1)
    code, flags = b.check_status()
    assert code == 5 and flags[0] & 1


def test_bounded_wait_gives_up_with_status(monkeypatch):
    """G2P waits on its staged bulk copies with a bounded number of polls.  The test-only
    MPM_TEST_G2P_WAIT_POLLS=0 makes that first wait give up at once (the copies themselves are
    ordinary and complete; the CTA's thread 0 waits for them, again bounded, before the CTA
    returns), so every staged chunk sets MPM_FLAG_WAIT and skips its work, and the host reads
    MPM_ERR_TIMEOUT.  A context created without the option then runs oracle-correct."""
    import torch

    from paper_2412_12089_gb300.batch import Batch

    # two substeps: G2P of substep 0 reads through the binning permutation (no staging); the
    # staged G2P of substep 1 is the step's last particle kernel, so the skipped chunks' state
    # is read only by the reward and get_state
    w = small("fluid", seed=9, substeps=2, T=1, n_envs=2, n=1500)
    monkeypatch.setenv("MPM_TEST_G2P_WAIT_POLLS", "0")
    b = Batch(w.specs, max_steps=0)
    monkeypatch.delenv("MPM_TEST_G2P_WAIT_POLLS")
    b.set_inits(w.inits)
    b.step(torch.as_tensor(w.actions[0]).cuda())
    code, flags = b.check_status()
    b.close()
    assert code == 6, code  # MPM_ERR_TIMEOUT
    assert all(f & 0x8 for f in flags), flags  # MPM_FLAG_WAIT in every env
    b2, rew, st = gpu_run(w, 1)
    code2, flags2 = b2.check_status()
    assert code2 == 0 and not flags2.any()
    for e in range(w.n_envs):
        o, q, r = oracle_run(w, e, 1)
        for k in ("x", "v", "F"):
            assert rel_err(split(w, st[k])[e], getattr(o, k)) < 1e-4, (e, k)
    b2.close()


# ------------------------------------------------------------------ gradients

def _gpu_grads(w, T, xbT=None, rbar=None, S=None):
    import torch

    from paper_2412_12089_gb300.batch import Batch

    b = Batch(w.specs, max_steps=T)
    b.set_inits(w.inits)
    for t in range(T):
        b.step(torch.as_tensor(w.actions[t]).cuda(), record=True)
    st = b.get_state()
    xb = None
    if xbT is not None:
        xb = xbT(st["x"].cpu().numpy())
    out = b.backward(xb=xb, reward_adj=rbar)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}, st


def test_gradient_cube_c1():
    """d/d(x0, v0, C0, F0) of sum |x_50 - x*|^2, x* = x0 + (0.05, 0, 0), on the full C1 cube."""
    w = wl.cube(seed=0)
    w.specs[0] = w.specs[0].replace(substeps=50)
    x0 = w.inits[0].x.astype(np.float64)
    target = x0 + np.array([0.05, 0.0, 0.0])
    g, st = _gpu_grads(w, 1, xbT=lambda xT: (2.0 * (xT - target)).astype(np.float32))
    s = w.specs[0]
    sp = orc.make_spec(s)
    so = orc.State.from_init(w.inits[0])
    oT, _, _ = oracle_run(w, 0, 1)
    ag, (xb, vb, Cb, Fb), qb = orc.rollout_adj(sp, so, np.zeros(4), np.zeros((1, 1)),
                                               adj_final=(2.0 * (oT.x - target), None, None, None))
    for name, got, ref in (("x", g["xb0"], xb), ("v", g["vb0"], vb), ("C", g["Cb0"], Cb), ("F", g["Fb0"], Fb)):
        assert rel_err(got, ref) < 1e-3, (name, rel_err(got, ref))


@pytest.mark.parametrize("name,S", [("dough", 4), ("fluid", 4), ("jumper", 3)])
def test_action_gradients(name, S):
    T = 2
    w = small(name, seed=9, substeps=S, T=T, n_envs=2)
    rbar = np.ones((T, w.n_envs), np.float32)
    g, st = _gpu_grads(w, T, rbar=rbar)
    for e in range(w.n_envs):
        s = w.specs[e]
        sp = orc.make_spec(s)
        so = orc.State.from_init(w.inits[e])
        A = s.action_dim
        ag, (xb, vb, Cb, Fb), qb = orc.rollout_adj(sp, so, orc.initial_pose(s),
                                                   w.actions[:T, e, :A].astype(np.float64), rbar=np.ones(T))
        assert rel_err(g["action_grad"][:, e, :A], ag) < 1e-3, (name, e, rel_err(g["action_grad"][:, e, :A], ag))
        assert rel_err(split(w, g["xb0"])[e], xb) < 1e-3, (name, e, "xb0")
        qb = qb.reshape(-1, 4).sum(0)  # gradient with respect to pose0 (capsule j at pose0 + j offset)
        assert rel_err(g["pose_grad0"][e], qb) < 1e-3 or np.abs(qb).max() < 1e-8, (name, e, g["pose_grad0"][e], qb)


def test_capsule_union_gradients():
    """Six independently driven capsules (24 collider actions per step): gradients of a loss on
    the final positions with respect to every capsule's actions, the initial state and pose0."""
    T = 2
    w = small("handflip", seed=12, substeps=4, T=T, n_envs=2)
    rng = np.random.default_rng(13)
    xw = rng.standard_normal((w.n_particles, 3)).astype(np.float32)
    g, st = _gpu_grads(w, T, xbT=lambda xT: xw)
    for e in range(w.n_envs):
        s = w.specs[e]
        sp = orc.make_spec(s)
        so = orc.State.from_init(w.inits[e])
        A = s.action_dim
        assert A == 24
        ag, (xb, vb, Cb, Fb), qb = orc.rollout_adj(sp, so, orc.initial_pose(s),
                                                   w.actions[:T, e, :A].astype(np.float64),
                                                   adj_final=(split(w, xw)[e].astype(np.float64), None, None, None))
        got = g["action_grad"][:, e, :A]
        assert rel_err(got, ag) < 1e-3, (e, rel_err(got, ag))
        # the contact is spread over the fingers: most capsules carry a gradient
        assert sum(np.abs(ag[:, 4 * j:4 * j + 4]).max() > 1e-6 * np.abs(ag).max() for j in range(6)) >= 4
        for name, gg, ref in (("x", g["xb0"], xb), ("v", g["vb0"], vb), ("F", g["Fb0"], Fb)):
            assert rel_err(split(w, gg)[e], ref) < 1e-3, (e, name, rel_err(split(w, gg)[e], ref))
        q4 = qb.reshape(-1, 4).sum(0)
        assert rel_err(g["pose_grad0"][e], q4) < 1e-3, (e, g["pose_grad0"][e], q4)


@pytest.mark.parametrize("tape_tiles", [None, "1", "300"])
def test_gradients_mixed_batch_grid_tape(tape_tiles, monkeypatch):
    """Environments of two materials and different substep counts reversed in one batch.
    The reverse pass restores the grids the recorded steps kept on the grid tape; with a
    one-tile pool no slot is kept and P2G rebuilds every grid, with a 300-tile pool the first
    substeps are kept and the rest rebuilt.  Either way each environment's gradients match its
    FP64 oracle."""
    if tape_tiles is not None:
        monkeypatch.setenv("MPM_GRID_TAPE_TILES", tape_tiles)
    T = 2
    d = small("dough", seed=12, substeps=5, T=T, n_envs=2, n_range=(500, 2000))
    f = small("fluid", seed=13, substeps=3, T=T, n_envs=1, n=1000)
    specs, inits = d.specs + f.specs, d.inits + f.inits
    A = max(s.action_dim for s in specs)
    acts = np.zeros((T, 3, A), np.float32)
    acts[:, :2, :d.actions.shape[2]] = d.actions[:T]
    acts[:, 2:, :f.actions.shape[2]] = f.actions[:T]
    w = wl.Workload("mixed", specs, inits, acts, T)
    g, _ = _gpu_grads(w, T, rbar=np.ones((T, 3), np.float32))
    for e in range(3):
        s = w.specs[e]
        sp = orc.make_spec(s)
        so = orc.State.from_init(w.inits[e])
        Ae = s.action_dim
        ag, (xb, vb, Cb, Fb), qb = orc.rollout_adj(sp, so, np.array(s.pose0, np.float64),
                                                   w.actions[:T, e, :Ae].astype(np.float64), rbar=np.ones(T))
        assert rel_err(g["action_grad"][:, e, :Ae], ag) < 1e-3, (e, rel_err(g["action_grad"][:, e, :Ae], ag))
        assert rel_err(split(w, g["xb0"])[e], xb) < 1e-3, (e, "xb0")
        assert rel_err(split(w, g["vb0"])[e], vb) < 1e-3, (e, "vb0")


@pytest.mark.parametrize("box", ["512", "1024", "256"])
def test_scatter_box_builds_match_oracle(box, monkeypatch):
    """Every scatter shape (512- and 1024-cell counting sorts on 256-particle four-warp CTAs,
    the 256-cell sort on 64-particle one-warp CTAs) of the scatter kernels (P2G forward, G2P^T
    in reverse) gives the oracle's substep and gradients."""
    monkeypatch.setenv("MPM_SCATTER_BOX", box)
    T = 1
    w = small("dough", seed=15, substeps=3, T=T, n_envs=2, n_range=(500, 3000))
    g, st = _gpu_grads(w, T, rbar=np.ones((T, w.n_envs), np.float32))
    for e in range(w.n_envs):
        s = w.specs[e]
        sp = orc.make_spec(s)
        so = orc.State.from_init(w.inits[e])
        A = s.action_dim
        o, _, _, _ = orc.rollout(sp, so, np.array(s.pose0, np.float64), w.actions[:T, e, :A].astype(np.float64))
        assert rel_err(split(w, st["x"].cpu().numpy())[e], o.x) < 1e-4  # three substeps
        ag, (xb, vb, Cb, Fb), qb = orc.rollout_adj(sp, so, np.array(s.pose0, np.float64),
                                                   w.actions[:T, e, :A].astype(np.float64), rbar=np.ones(T))
        assert rel_err(g["action_grad"][:, e, :A], ag) < 1e-3


@pytest.mark.parametrize("box", ["512", "256"])
def test_sparse_cloud_groups_by_runs(box, monkeypatch):
    """Particles scattered thinly (about 0.1 per cell) over most of the domain, so a chunk's
    cells outnumber its counting sort's capacity and the scatter kernels group the chunk by
    runs of equal cell base in binned order instead, marking tiles per run: two substeps and
    the gradient of sum |x_T - x*|^2 against the oracle."""
    monkeypatch.setenv("MPM_SCATTER_BOX", box)
    n = 1500
    w = small("cube", seed=21, n=n, G=32, substeps=2, T=1)
    rng = np.random.default_rng(21)
    w.inits[0].x = (0.15 + 0.7 * rng.random((n, 3))).astype(np.float32)
    w = perturb(w, seed=22)
    x0 = w.inits[0].x.astype(np.float64)
    target = x0 + np.array([0.02, 0.0, 0.0])
    g, st = _gpu_grads(w, 1, xbT=lambda xT: (2.0 * (xT - target)).astype(np.float32))
    oT, _, _ = oracle_run(w, 0, 1)
    xs = st["x"].cpu().numpy()
    assert rel_err(xs, oT.x) < 1e-4, rel_err(xs, oT.x)  # two substeps
    sp = orc.make_spec(w.specs[0])
    so = orc.State.from_init(w.inits[0])
    ag, (xb, vb, Cb, Fb), qb = orc.rollout_adj(sp, so, np.zeros(4), np.zeros((1, 1)),
                                               adj_final=(2.0 * (oT.x - target), None, None, None))
    for name, got, ref in (("x", g["xb0"], xb), ("v", g["vb0"], vb), ("C", g["Cb0"], Cb), ("F", g["Fb0"], Fb)):
        assert rel_err(got, ref) < 1e-3, (name, rel_err(got, ref))


def test_autotune_picks_a_box_and_keeps_results():
    import torch

    from paper_2412_12089_gb300 import mpm
    from paper_2412_12089_gb300.batch import Batch

    w = small("dough", seed=14, substeps=3, T=2, n_envs=3, n_range=(500, 4000))
    _, rew0, st0 = gpu_run(w, 2)
    b = Batch(w.specs, max_steps=0)
    b.set_inits(w.inits)
    stage0 = mpm.mpm_autotune_config(b.ctx)["g2p_stage"]
    chosen, times = mpm.mpm_autotune(b.ctx, trials=2)
    assert set(chosen) == {"vonmises"} and chosen["vonmises"] in (512, 1024, 256)
    assert all(t > 0 for trio in times.values() for t in trio)
    assert chosen["vonmises"] == (512, 1024, 256)[int(np.argmin(times["vonmises"]))]
    cfg = mpm.mpm_autotune_config(b.ctx)
    assert cfg["grid_blocks"] in (304, 608, 1216, 2432)
    assert cfg["grid_blocks"] == (304, 608, 1216, 2432)[int(np.argmin(cfg["grid_ms_304_608_1216_2432"]))]
    assert cfg["g2p_stage"] == stage0  # no tape: G2P staging is not tuned, it keeps its value
    rews = [b.step(torch.as_tensor(w.actions[t]).cuda()).clone() for t in range(2)]
    st = {k: v.cpu().numpy() for k, v in b.get_state().items()}
    assert rel_err(st["x"], st0["x"]) < 1e-5  # the tuning trials left the state unchanged
    assert np.allclose(torch.stack(rews).cpu().numpy(), rew0, rtol=1e-5, atol=1e-7)
    with pytest.raises(mpm.MpmError):
        mpm.mpm_autotune(b.ctx, trials=0)
    # with a checkpoint tape the G2P staging is tuned as well, on the ring's first block,
    # and the recorded steps and their gradients are unchanged by the trials
    bt = Batch(w.specs, max_steps=2)
    bt.set_inits(w.inits)
    # a context built after a tuning starts from its choices (kept for the process: the
    # grid kernels' CTA count, and per material, grid resolution and particles-per-cell
    # bucket the scatter shape and G2P staging)
    assert mpm.mpm_autotune_config(bt.ctx)["grid_blocks"] == cfg["grid_blocks"]
    mpm.mpm_autotune(bt.ctx, trials=2)
    cfg = mpm.mpm_autotune_config(bt.ctx)
    plain, staged = cfg["g2p_ms_plain_staged"]["vonmises"]
    assert plain > 0 and staged > 0 and cfg["g2p_stage"]["vonmises"] == (0 if plain < staged else 1)
    rews_t = [bt.step(torch.as_tensor(w.actions[t]).cuda(), record=True).clone() for t in range(2)]
    st_t = {k: v.cpu().numpy() for k, v in bt.get_state().items()}
    assert rel_err(st_t["x"], st0["x"]) < 1e-5
    assert np.allclose(torch.stack(rews_t).cpu().numpy(), rew0, rtol=1e-5, atol=1e-7)
    bt.close()
