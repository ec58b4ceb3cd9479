"""Shared helpers of the GPU parity tests: run a workload through the C ABI and
through the FP64 oracle on the same FP32 inputs."""
from __future__ import annotations

import numpy as np

from oracle import oracle as orc
from paper_2412_12089_gb300 import workloads as wl


def rel_err(a, b):
    """infinity-norm relative error |a - b|_inf / max(|b|_inf, 1e-12)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-12))


def perturb(w: wl.Workload, seed=0, F_std=0.04, C_std=0.5, v_std=0.3):
    """Give a workload a non-trivial FP32 start state (deformed F, non-zero C and v) so one
    substep exercises every term of the stress, the return mapping and APIC."""
    rng = np.random.default_rng(seed)
    for s, i in zip(w.specs, w.inits):
        n = s.n_particles
        i.v = (i.v + v_std * rng.standard_normal((n, 3))).astype(np.float32)
        i.C = (C_std * rng.standard_normal((n, 3, 3))).astype(np.float32)
        if s.material == "fluid":
            J = 1.0 + 0.02 * rng.standard_normal((n, 1, 1))
            i.F = (np.cbrt(J) * np.eye(3)).astype(np.float32)
        else:
            i.F = (np.eye(3) + F_std * rng.standard_normal((n, 3, 3))).astype(np.float32)
    return w


def gpu_run(w: wl.Workload, T: int, record=False, use_graphs=True, per_env=False, max_steps=None):
    """Run T control steps of the workload on the GPU; return (batch, rewards [T, n_envs],
    final state dict of numpy arrays)."""
    import torch

    from paper_2412_12089_gb300.batch import Batch

    b = Batch(w.specs, max_steps=(T if max_steps is None else max_steps) if record else 0, per_env_launch=per_env,
              use_graphs=use_graphs)
    b.set_inits(w.inits)
    rews = []
    for t in range(T):
        rews.append(b.step(torch.as_tensor(w.actions[t]).cuda(), record=record).clone())
    st = b.get_state()
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in st.items()}
    return b, torch.stack(rews).cpu().numpy(), out


def split(w: wl.Workload, arr):
    offs = np.cumsum([0] + [s.n_particles for s in w.specs])
    return [arr[offs[e]:offs[e + 1]] for e in range(w.n_envs)]


def oracle_run(w: wl.Workload, e: int, T: int):
    s = w.specs[e]
    sp = orc.make_spec(s)
    st = orc.State.from_init(w.inits[e])
    A = s.action_dim
    acts = w.actions[:T, e, :max(A, 1)].astype(np.float64)
    out, q, rew, status = orc.rollout(sp, st, orc.initial_pose(s), acts)
    return out, q, rew


def oracle_pool(n_jobs):
    """A process pool for oracle runs, started with spawn (safe after CUDA is initialised)."""
    import multiprocessing as mp
    import os

    return mp.get_context("spawn").Pool(max(1, min(n_jobs, len(os.sched_getaffinity(0)))))


def oracle_trajectory(job):
    """Pool worker: the oracle's state after each of T control steps of env e of a workload
    (rebuilt from its maker and keyword arguments).  Returns (e, [(x, v, C, F)] * T, rewards)."""
    maker, kw, e, T = job
    w = getattr(wl, maker)(**kw)
    s = w.specs[e]
    sp = orc.make_spec(s)
    st = orc.State.from_init(w.inits[e])
    acts = w.actions[:T, e, :max(s.action_dim, 1)].astype(np.float64)
    q = orc.initial_pose(s)
    traj, rews = [], []
    for t in range(T):
        st, q, r, _ = orc.rollout(sp, st, q, acts[t:t + 1])
        traj.append((st.x.copy(), st.v.copy(), st.C.copy(), st.F.copy()))
        rews.append(r[0])
    return e, traj, np.array(rews)


def final_adjoint(w, e):
    """A seeded adjoint of the final positions (the loss sum_p xbar_p . x_p), env e."""
    return np.random.default_rng(100 + e).standard_normal((w.specs[e].n_particles, 3))


def oracle_gradients(job):
    """Pool worker: the oracle's gradients of sum_t r_t + sum_p xbar_p . x_p(T) for env e:
    (e, action gradient (T, A), (xb0, vb0, Cb0, Fb0))."""
    maker, kw, e, T = job
    w = getattr(wl, maker)(**kw)
    s = w.specs[e]
    sp = orc.make_spec(s)
    st = orc.State.from_init(w.inits[e])
    acts = w.actions[:T, e, :max(s.action_dim, 1)].astype(np.float64)
    ag, sb, _ = orc.rollout_adj(sp, st, orc.initial_pose(s), acts, adj_final=(final_adjoint(w, e), None, None, None),
                                rbar=np.ones(T))
    return e, ag, sb


def oracle_return(job):
    """Pool worker: the oracle's total reward sum_t r_t of env e over T control steps, with
    action entry (t, j) shifted by h (t < 0: no shift).  For central differences."""
    maker, kw, e, T, t, j, h = job
    w = getattr(wl, maker)(**kw)
    s = w.specs[e]
    sp = orc.make_spec(s)
    st = orc.State.from_init(w.inits[e])
    acts = w.actions[:T, e, :max(s.action_dim, 1)].astype(np.float64)
    if t >= 0:
        acts[t, j] += h
    _, _, rew, status = orc.rollout(sp, st, orc.initial_pose(s), acts)
    return float(rew.sum()), int(status)
