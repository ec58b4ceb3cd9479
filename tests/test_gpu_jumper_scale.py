"""Differentiation at scale: the soft jumper (App. E's SoftJumper recast as MPM: muscle legs
with an active fibre stress per actuator group, a passive neo-Hookean torso, ground contact
with friction) over its full horizon of 64 control steps x 20 substeps, every control step
checkpointed and the whole horizon reversed (Sec. 4.1).

  - 64 envs x 100k particles on 96^3 grids, in one batch: recorded and reversed end to end.
    Sampled environments are checked against the FP64 oracle over the first two control
    steps (state and rewards), and their action gradients of the last two control steps
    against the oracle's exact adjoint started from the GPU's own checkpoint of that state
    (the reward sum's gradient with respect to a_62 and a_63 depends on nothing earlier).
  - A reduced jumper (4,500 particles on 48^3, the same 222 groups and constants) over the
    same 64 x 20 horizon: the GPU's FP32 gradient of sum_t r_t with respect to 16 seeded
    action coordinates against FP64 central differences of the oracle's forward rollouts.

Tolerances: 1e-3 (infinity-norm relative) on states, rewards and gradients.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2412_12089_gb300 import workloads as wl

from gpu_helpers import oracle_pool, oracle_return, rel_err, split

pytestmark = pytest.mark.gpu

T_FULL = 64


def _oracle_first_steps(job):
    e, T = job
    w = wl.jumper(n_envs=64, seed=0, T=T_FULL)
    s = w.specs[e]
    out, q, r, status = orc.rollout(orc.make_spec(s), orc.State.from_init(w.inits[e]), orc.initial_pose(s),
                                    w.actions[:T, e, :s.action_dim].astype(np.float64))
    return e, out, r, status


def _oracle_tail_grad(job):
    e, t0, x, v, C, F, group = job
    w = wl.jumper(n_envs=64, seed=0, T=T_FULL)
    s = w.specs[e]
    st = orc.State(x, v, C, F, group)
    acts = w.actions[t0:T_FULL, e, :s.action_dim].astype(np.float64)
    ag, _, _ = orc.rollout_adj(orc.make_spec(s), st, orc.initial_pose(s), acts, rbar=np.ones(T_FULL - t0))
    return e, ag


def test_jumper_64x100k_full_horizon_record_and_reverse():
    import torch

    from paper_2412_12089_gb300 import mpm
    from paper_2412_12089_gb300.batch import Batch

    w = wl.jumper(n_envs=64, seed=0, T=T_FULL)
    sample = (0, 37)
    T_head, t_tail = 2, T_FULL - 2
    pool = oracle_pool(2 * len(sample))
    try:
        head = pool.map_async(_oracle_first_steps, [(e, T_head) for e in sample])
        b = Batch(w.specs, max_steps=T_FULL)
        b.set_inits(w.inits)
        acts = torch.as_tensor(w.actions).cuda()
        rews = []
        tail_jobs = []
        for t in range(T_FULL):
            if t == t_tail:
                st = {k: v.cpu().numpy().astype(np.float64) for k, v in b.get_state().items()}
                for e in sample:
                    tail_jobs.append((e, t_tail, split(w, st["x"])[e], split(w, st["v"])[e], split(w, st["C"])[e],
                                      split(w, st["F"])[e], w.inits[e].group))
                tail = pool.map_async(_oracle_tail_grad, tail_jobs)
            rews.append(b.step(acts[t], record=True).cpu().numpy())
            if t + 1 == T_head:
                head_state = {k: v.cpu().numpy() for k, v in b.get_state().items()}
        assert b.tape_length() == T_FULL
        g = b.backward(reward_adj=torch.ones(T_FULL, w.n_envs, device="cuda"), want_state=False)
        agrad = g["action_grad"].cpu().numpy()
        code, flags = b.check_status()
        gb = mpm.mpm_device_bytes(b.ctx) / 1e9
        b.close()
        heads = head.get()
        tails = tail.get()
    finally:
        pool.close()
        pool.join()
    print(f"\njumper 64 x 100k, {T_FULL} x 20 recorded and reversed: {gb:.1f} GB on the device")
    assert code == 0 and not flags.any()
    assert np.isfinite(agrad).all() and np.abs(agrad).max() > 0
    rews = np.array(rews)
    for e, out, r, status in heads:
        assert status == 0
        for k in ("x", "v", "F"):
            err = rel_err(split(w, head_state[k])[e], getattr(out, k))
            print(f"env {e}: {k} after {T_head} control steps {err:.2e}")
            assert err < 1e-3, (e, k, err)
        assert np.allclose(rews[:T_head, e], r, rtol=1e-3, atol=1e-6), (e, rews[:T_head, e], r)
    for e, ag in tails:
        A = w.specs[e].action_dim
        err = rel_err(agrad[t_tail:, e, :A], ag)
        print(f"env {e}: action gradient of control steps {t_tail}..{T_FULL - 1} {err:.2e}")
        assert err < 1e-3, (e, err)


def test_jumper_gradient_vs_central_differences_full_horizon():
    """FP32 reverse pass through 64 recorded control steps vs FP64 central differences."""
    import torch

    from paper_2412_12089_gb300.batch import Batch

    kw = dict(n_envs=1, seed=4, n=4500, G=48, T=T_FULL)
    w = wl.jumper(**kw)
    A = w.specs[0].action_dim
    rng = np.random.default_rng(16)
    coords = [(int(rng.integers(0, T_FULL)), int(rng.integers(0, A))) for _ in range(16)]
    h = 1e-4  # FP64 central differences of the oracle agree with its adjoint to 4e-8 here
    jobs = [("jumper", kw, 0, T_FULL, t, j, s * h) for (t, j) in coords for s in (1.0, -1.0)]
    pool = oracle_pool(len(jobs))
    try:
        pending = pool.map_async(oracle_return, jobs)
        b = Batch(w.specs, max_steps=T_FULL)
        b.set_inits(w.inits)
        for t in range(T_FULL):
            b.step(torch.as_tensor(w.actions[t]).cuda(), record=True)
        g = b.backward(reward_adj=torch.ones(T_FULL, 1, device="cuda"), want_state=False)
        agrad = g["action_grad"].cpu().numpy()[:, 0, :A]
        code, flags = b.check_status()
        b.close()
        res = pending.get()
    finally:
        pool.close()
        pool.join()
    assert code == 0 and not flags.any()
    assert all(st == 0 for _, st in res)
    fd = np.array([(res[2 * i][0] - res[2 * i + 1][0]) / (2 * h) for i in range(len(coords))])
    gpu = np.array([agrad[t, j] for t, j in coords])
    err = float(np.abs(gpu - fd).max() / np.abs(fd).max())
    for (t, j), a, f in zip(coords, gpu, fd):
        print(f"a[{t:2d}, {j:3d}]: gpu {a:+.6e}  fd {f:+.6e}")
    print(f"max relative error {err:.2e}")
    assert err < 1e-3, err
