"""Tetrahedral-FEM environments (App. D.2 stable neo-Hookean elements; App. E SoftJumper) on
the CUDA path against the FP64 FEM oracle:

- one substep from a deformed, moving state with ground contact (1e-5);
- a 2-control-step horizon of the SoftJumper batch at its 80 substeps per step (1e-3);
- gradients of rewards plus a loss on the final positions with respect to all actions and
  the initial state (1e-3), with and without ground contact;
- FEM and MPM environments mixed in one batch, forward and reverse, each against its own
  oracle, and bitwise equal to the per-environment launch path for the FEM environment;
- the smallest meshes (one element, one voxel) beside the largest element count the ABI takes
  (1,020 of 1,024), forward and reverse.
"""
import numpy as np
import pytest

from oracle import fem
from oracle import oracle as orc
from paper_2412_12089_gb300 import workloads as wl

from gpu_helpers import rel_err, split

pytestmark = pytest.mark.gpu


def jumpers(n_envs=3, seed=0, substeps=80, T=2, ground=None, v_std=0.0, jitter=0.0):
    """SoftJumper batch; ground: height of the ground above each body's lowest vertex (None: far
    below, no contact)."""
    w = wl.softjumper(n_envs=n_envs, seed=seed, substeps=substeps, T=T)
    rng = np.random.default_rng(seed + 100)
    for e in range(n_envs):
        i = w.inits[e]
        if jitter:
            i.x = (i.x + jitter * rng.standard_normal(i.x.shape)).astype(np.float32)
        if v_std:
            i.v = (v_std * rng.standard_normal(i.v.shape)).astype(np.float32)
        gz = -1.0 if ground is None else float(i.x[:, 2].min()) + ground
        w.specs[e] = w.specs[e].replace(ground_z=float(np.float32(gz)))
    return w


def run_gpu(w, T, record=False):
    import torch

    from paper_2412_12089_gb300.batch import Batch

    b = Batch(w.specs, max_steps=T if record else 0)
    b.set_inits(w.inits)
    rew = [b.step(torch.as_tensor(w.actions[t]).cuda(), record=record).clone() for t in range(T)]
    st = {k: v.cpu().numpy() for k, v in b.get_state().items()}
    return b, torch.stack(rew).cpu().numpy(), st


def fem_oracle(w, e, T):
    s = w.specs[e]
    m = fem.make_mesh(s)
    x, v, r, st = fem.rollout(m, w.inits[e].x, w.inits[e].v, w.actions[:T, e, :s.n_groups])
    return x, v, r, st


def test_fem_substep_parity_with_ground():
    # one substep (of h = 1/60 s: a single step of the scheme, not a stable trajectory) from
    # jittered (stressed), moving bodies, the lowest vertices on the ground
    w = jumpers(n_envs=3, seed=1, substeps=1, T=1, ground=0.004, v_std=0.5, jitter=0.002)
    b, rew, st = run_gpu(w, 1)
    try:
        code, flags = b.check_status()
    finally:
        b.close()
    assert code == 0 and not flags.any()
    for e in range(w.n_envs):
        x, v, r, _ = fem_oracle(w, e, 1)
        assert (w.inits[e].x[:, 2] <= w.specs[e].ground_z).sum() >= 3
        assert rel_err(split(w, st["x"])[e], x) < 1e-5, (e, rel_err(split(w, st["x"])[e], x))
        assert rel_err(split(w, st["v"])[e], v) < 1e-5, (e, rel_err(split(w, st["v"])[e], v))
        assert abs(rew[0, e] - r[0]) <= 1e-5 * max(1.0, abs(r[0]))
        assert np.all(split(w, st["C"])[e] == 0.0)


def test_fem_horizon_parity_softjumper():
    w = jumpers(n_envs=4, seed=2, substeps=80, T=2)
    b, rew, st = run_gpu(w, 2)
    b.close()
    for e in range(w.n_envs):
        x, v, r, status = fem_oracle(w, e, 2)
        assert status == 0
        assert rel_err(split(w, st["x"])[e], x) < 1e-3, (e, rel_err(split(w, st["x"])[e], x))
        assert rel_err(split(w, st["v"])[e], v) < 1e-3, (e, rel_err(split(w, st["v"])[e], v))
        assert np.allclose(rew[:, e], r, rtol=1e-3, atol=1e-5), (e, rew[:, e], r)


@pytest.mark.parametrize("ground", [None, 0.004])
def test_fem_gradients_match_oracle(ground):
    import torch

    from paper_2412_12089_gb300.batch import Batch

    T = 2
    # 80 substeps keep the explicit scheme's dt = 1/4800 s inside its stability limit
    w = jumpers(n_envs=2, seed=3, substeps=80, T=T, ground=ground, v_std=0.2, jitter=0.001)
    rng = np.random.default_rng(5)
    xw = rng.standard_normal((w.n_particles, 3)).astype(np.float32)
    rbar = rng.standard_normal((T, w.n_envs)).astype(np.float32)
    b = Batch(w.specs, max_steps=T)
    try:
        b.set_inits(w.inits)
        for t in range(T):
            b.step(torch.as_tensor(w.actions[t]).cuda(), record=True)
        g = {k: v.cpu().numpy() for k, v in b.backward(xb=xw, reward_adj=rbar).items()}
    finally:
        b.close()
    for e in range(w.n_envs):
        s = w.specs[e]
        m = fem.make_mesh(s)
        A = s.n_groups
        ag, xb, vb, _ = fem.rollout_adj(m, w.inits[e].x, w.inits[e].v, w.actions[:T, e, :A],
                                        xbT=split(w, xw)[e], rbar=rbar[:, e])
        assert rel_err(g["action_grad"][:, e, :A], ag) < 1e-3, (e, rel_err(g["action_grad"][:, e, :A], ag))
        assert rel_err(split(w, g["xb0"])[e], xb) < 1e-3, (e, "xb0", rel_err(split(w, g["xb0"])[e], xb))
        assert rel_err(split(w, g["vb0"])[e], vb) < 1e-3, (e, "vb0", rel_err(split(w, g["vb0"])[e], vb))


def test_fem_and_mpm_in_one_batch():
    import torch

    from paper_2412_12089_gb300.batch import Batch

    T = 2
    j = jumpers(n_envs=1, seed=4, substeps=80, T=T, v_std=0.1)
    f = wl.fluid(n_envs=1, seed=44, n=900, substeps=3, T=T)
    specs, inits = j.specs + f.specs, j.inits + f.inits
    A = max(s.action_dim for s in specs)
    acts = np.zeros((T, 2, A), np.float32)
    acts[:, :1, :j.actions.shape[2]] = j.actions[:T]
    acts[:, 1:, :f.actions.shape[2]] = f.actions[:T]
    w = wl.Workload("mixed", specs, inits, acts, T)
    rbar = np.ones((T, 2), np.float32)
    b = Batch(w.specs, max_steps=T)
    try:
        b.set_inits(w.inits)
        rew = [b.step(torch.as_tensor(acts[t]).cuda(), record=True).clone() for t in range(T)]
        st = {k: v.cpu().numpy() for k, v in b.get_state().items()}
        g = {k: v.cpu().numpy() for k, v in b.backward(reward_adj=rbar).items()}
        rew = torch.stack(rew).cpu().numpy()
    finally:
        b.close()
    # the FEM kernels sum in a fixed order: the per-env launch path gives identical bits
    bp = Batch(w.specs, max_steps=T, per_env_launch=True, use_graphs=False)
    try:
        bp.set_inits(w.inits)
        for t in range(T):
            bp.step(torch.as_tensor(acts[t]).cuda(), record=True)
        stp = {k: v.cpu().numpy() for k, v in bp.get_state().items()}
        gp = {k: v.cpu().numpy() for k, v in bp.backward(reward_adj=rbar).items()}
    finally:
        bp.close()
    assert np.array_equal(split(w, stp["x"])[0], split(w, st["x"])[0])
    assert np.array_equal(gp["action_grad"][:, 0], g["action_grad"][:, 0])
    # FEM env
    s0 = specs[0]
    m = fem.make_mesh(s0)
    x, v, r, _ = fem.rollout(m, inits[0].x, inits[0].v, acts[:T, 0, :s0.n_groups])
    assert rel_err(split(w, st["x"])[0], x) < 1e-3 and np.allclose(rew[:, 0], r, rtol=1e-3, atol=1e-5)
    ag, xb, vb, _ = fem.rollout_adj(m, inits[0].x, inits[0].v, acts[:T, 0, :s0.n_groups], rbar=np.ones(T))
    assert rel_err(g["action_grad"][:, 0, :s0.n_groups], ag) < 1e-3
    assert rel_err(split(w, g["xb0"])[0], xb) < 1e-3
    # fluid env
    s1 = specs[1]
    sp = orc.make_spec(s1)
    so = orc.State.from_init(inits[1])
    A1 = s1.action_dim
    out, q, r1, _ = orc.rollout(sp, so, orc.initial_pose(s1), acts[:T, 1, :A1].astype(np.float64))
    assert rel_err(split(w, st["x"])[1], out.x) < 1e-3
    ag1, (xb1, _, _, _), _ = orc.rollout_adj(sp, so, orc.initial_pose(s1), acts[:T, 1, :A1].astype(np.float64),
                                             rbar=np.ones(T))
    assert rel_err(g["action_grad"][:, 1, :A1], ag1) < 1e-3
    assert rel_err(split(w, g["xb0"])[1], xb1) < 1e-3


def fem_body(tets, rest, n_act, substeps=80, ground_z=-1.0):
    """A SoftJumper-like FEM environment (same material, damping and reward) on any mesh."""
    n, n_t = rest.shape[0], tets.shape[0]
    group = (np.arange(n_t) * n_act // n_t).astype(np.int32)
    h0 = float(np.float32(rest[:, 2].astype(np.float64).mean()))
    return wl.EnvSpec(n_particles=n, grid_res=8, substeps=substeps, dt=(1.0 / 60.0) / substeps, material="fem",
                      E=2500.0, nu=0.25, rho=1.0, act_stress=0.2, n_groups=n_act, ground_mu=0.5, reward="jump",
                      n_sub=n, rparam=(h0, 3.0, 1e-4, 0.0), k_damp=1.0, ground_z=float(np.float32(ground_z)),
                      fem_tets=tets, fem_rest=rest, fem_group=group, bound=0)


def tiny_and_largest_meshes(T, seed=21):
    rng = np.random.default_rng(seed)
    one = np.array([[0.5, 0.5, 0.5], [0.55, 0.5, 0.5], [0.5, 0.55, 0.5], [0.5, 0.5, 0.55]], np.float32)
    vox_rest, vox_tets = wl.voxel_mesh(np.ones((1, 1, 1), bool), 0.05, origin=(0.45, 0.45, 0.3))
    slab_rest, slab_tets = wl.voxel_mesh(np.ones((12, 17, 1), bool), 0.05, origin=(0.2, 0.075, 0.2))
    assert slab_tets.shape[0] == 1020
    specs = [fem_body(np.array([[0, 1, 2, 3]], np.int32), one, 1),
             fem_body(vox_tets, vox_rest, 2, ground_z=float(vox_rest[:, 2].min()) + 0.004),
             fem_body(slab_tets, slab_rest, 255)]
    inits = []
    for sp in specs:
        v = (0.1 * rng.standard_normal((sp.n_particles, 3))).astype(np.float32)
        inits.append(wl.EnvInit(sp.fem_rest.copy(), v, np.zeros((sp.n_particles, 3, 3), np.float32),
                                np.broadcast_to(np.eye(3, dtype=np.float32), (sp.n_particles, 3, 3)).copy()))
    acts = np.zeros((T, 3, 255), np.float32)
    for e, sp in enumerate(specs):
        acts[:, e, :sp.n_groups] = rng.uniform(-1.0, 1.0, (T, sp.n_groups))
    return wl.Workload("fem-sizes", specs, inits, acts, T)


def test_fem_smallest_and_largest_meshes():
    import torch

    from paper_2412_12089_gb300.batch import Batch

    T = 2
    w = tiny_and_largest_meshes(T)
    rng = np.random.default_rng(22)
    xw = rng.standard_normal((w.n_particles, 3)).astype(np.float32)
    rbar = rng.standard_normal((T, w.n_envs)).astype(np.float32)
    b = Batch(w.specs, max_steps=T)
    try:
        b.set_inits(w.inits)
        rew = [b.step(torch.as_tensor(w.actions[t]).cuda(), record=True).clone() for t in range(T)]
        st = {k: v.cpu().numpy() for k, v in b.get_state().items()}
        g = {k: v.cpu().numpy() for k, v in b.backward(xb=xw, reward_adj=rbar).items()}
        code, flags = b.check_status()
        rew = torch.stack(rew).cpu().numpy()
    finally:
        b.close()
    assert code == 0 and not flags.any()
    for e in range(w.n_envs):
        s = w.specs[e]
        m = fem.make_mesh(s)
        A = s.n_groups
        x, v, r, status = fem.rollout(m, w.inits[e].x, w.inits[e].v, w.actions[:T, e, :A])
        assert status == 0
        assert rel_err(split(w, st["x"])[e], x) < 1e-3, (e, rel_err(split(w, st["x"])[e], x))
        assert rel_err(split(w, st["v"])[e], v) < 1e-3, (e, rel_err(split(w, st["v"])[e], v))
        assert np.allclose(rew[:, e], r, rtol=1e-3, atol=1e-5), (e, rew[:, e], r)
        ag, xb, vb, _ = fem.rollout_adj(m, w.inits[e].x, w.inits[e].v, w.actions[:T, e, :A],
                                        xbT=split(w, xw)[e], rbar=rbar[:, e])
        assert rel_err(g["action_grad"][:, e, :A], ag) < 1e-3, (e, rel_err(g["action_grad"][:, e, :A], ag))
        assert rel_err(split(w, g["xb0"])[e], xb) < 1e-3, (e, "xb0", rel_err(split(w, g["xb0"])[e], xb))
        assert rel_err(split(w, g["vb0"])[e], vb) < 1e-3, (e, "vb0", rel_err(split(w, g["vb0"])[e], vb))
