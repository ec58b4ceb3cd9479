"""Torch-facing wrapper of a batch context: device memory and streams come from
PyTorch, every simulation step runs in libmpm_gb300.so through the C ABI.

``Batch`` holds one mpm_ctx (many environments stepped together).  ``MPMRollout`` is
the custom autograd Function of the paper's Sec. 4.1: its forward records a rollout
on the checkpoint tape, its backward runs the library's reverse pass (checkpoint
restore + substep recomputation + adjoint kernels) and returns the gradients with
respect to the actions and the initial state.
"""
from __future__ import annotations

import numpy as np

from . import mpm


def _torch():
    import torch

    return torch


class Batch:
    def __init__(self, specs, max_steps=0, per_env_launch=False, use_graphs=True, device=0, keep_fraction=0.0):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("Batch needs a CUDA device")
        self.specs = list(specs)
        self.device = torch.device("cuda", device)
        self.ctx = mpm.mpm_create(self.specs, max_steps=max_steps, per_env_launch=per_env_launch,
                                  use_graphs=use_graphs, device=device, keep_fraction=keep_fraction)
        L = mpm.lib()
        self.n_envs = L.mpm_n_envs(self.ctx)
        self.P = L.mpm_n_particles(self.ctx)
        self.A = L.mpm_action_dim(self.ctx)
        self.max_steps = max_steps
        self.counts = [s.n_particles for s in self.specs]

    def close(self):
        if getattr(self, "ctx", None):
            mpm.mpm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, a, dtype=None):
        torch = _torch()
        dtype = dtype or torch.float32
        if a is None:
            return None
        t = torch.as_tensor(a, dtype=dtype, device=self.device)
        return t.contiguous()

    def set_state(self, x, v, C, F, group=None, pose=None):
        torch = _torch()
        args = [self._dev(a) for a in (x, v, C, F)]
        g = self._dev(group, torch.int32) if group is not None else None
        p = self._dev(pose) if pose is not None else None
        mpm.mpm_set_state(self.ctx, *args, group=g, pose=p)
        self._keep = (args, g, p)  # alive until the stream has consumed them

    def set_inits(self, inits, poses=None):
        x = np.concatenate([i.x for i in inits])
        v = np.concatenate([i.v for i in inits])
        C = np.concatenate([i.C for i in inits])
        F = np.concatenate([i.F for i in inits])
        g = np.concatenate([i.group for i in inits])
        if poses is None:
            poses = np.array([s.pose0 for s in self.specs], np.float32)
        self.set_state(x, v, C, F, group=g, pose=poses)

    def get_state(self):
        torch = _torch()
        P = self.P
        out = {"x": torch.empty(P, 3, device=self.device), "v": torch.empty(P, 3, device=self.device),
               "C": torch.empty(P, 3, 3, device=self.device), "F": torch.empty(P, 3, 3, device=self.device),
               "pose": torch.empty(self.n_envs, 4, device=self.device)}
        mpm.mpm_get_state(self.ctx, out["x"], out["v"], out["C"], out["F"], out["pose"])
        return out

    def step(self, actions=None, record=False, reward=None):
        torch = _torch()
        a = None
        if actions is not None:
            a = self._dev(actions).reshape(self.n_envs, -1)
            if a.shape[1] != self.A:
                raise ValueError(f"actions must be [n_envs, {self.A}]")
        r = reward if reward is not None else torch.empty(self.n_envs, device=self.device)
        mpm.mpm_step(self.ctx, a, r, mpm.MPM_STEP_RECORD if record else 0)
        self._keep_a = a
        return r

    @property
    def obs_dim(self):
        return mpm.mpm_obs_dim(self.ctx)

    def observe(self):
        """Task observation of every env's current state: [n_envs, obs_dim] (x' zero padded,
        then the mean of x', 4 pose entries, 3 target entries)."""
        torch = _torch()
        out = torch.empty(self.n_envs, self.obs_dim, device=self.device)
        mpm.mpm_observe(self.ctx, out)
        return out

    def backward(self, xb=None, vb=None, Cb=None, Fb=None, reward_adj=None, want_state=True, obs_adj=None):
        """obs_adj: [T + 1, n_envs, obs_dim] adjoints of the observations of the recorded
        states (row t before step t, row T the final state), or None."""
        torch = _torch()
        T = mpm.mpm_tape_length(self.ctx)
        if obs_adj is not None:
            mpm.mpm_set_obs_adjoint(self.ctx, self._dev(obs_adj).contiguous())
        P = self.P
        out = {"action_grad": torch.empty(T, self.n_envs, self.A, device=self.device)}
        if want_state:
            out.update(xb0=torch.empty(P, 3, device=self.device), vb0=torch.empty(P, 3, device=self.device),
                       Cb0=torch.empty(P, 3, 3, device=self.device), Fb0=torch.empty(P, 3, 3, device=self.device),
                       pose_grad0=torch.empty(self.n_envs, 4, device=self.device))
        ins = [self._dev(a) for a in (xb, vb, Cb, Fb)]
        rb = self._dev(reward_adj)
        mpm.mpm_backward(self.ctx, *ins, reward_adj=rb, action_grad=out["action_grad"], xb0=out.get("xb0"),
                         vb0=out.get("vb0"), Cb0=out.get("Cb0"), Fb0=out.get("Fb0"),
                         pose_grad0=out.get("pose_grad0"))
        self._keep_b = (ins, rb)
        return out

    # step-wise reverse pass (closed-loop consumers): begin, one call per recorded step from
    # the last, end
    def backward_begin(self, xb=None, vb=None, Cb=None, Fb=None):
        ins = [self._dev(a) for a in (xb, vb, Cb, Fb)]
        mpm.mpm_backward_begin(self.ctx, *ins)
        self._keep_b = ins

    def backward_step(self, reward_adj=None, obs_adj=None):
        """Reverse the next recorded step t (the last first).  reward_adj: [n_envs] adjoint of
        r_t; obs_adj: [n_envs, obs_dim] adjoint of the observation of step t's end state.
        Returns (t, action_grad [n_envs, A]): the total adjoint of a_t."""
        torch = _torch()
        ag = torch.empty(self.n_envs, self.A, device=self.device)
        rb, ob = self._dev(reward_adj), self._dev(obs_adj)
        t = mpm.mpm_backward_step(self.ctx, reward_adj=rb, obs_adj=ob, action_grad=ag)
        self._keep_s = (rb, ob)
        return t, ag

    def backward_end(self, obs_adj=None, want_state=False):
        torch = _torch()
        P = self.P
        out = {"pose_grad0": torch.empty(self.n_envs, 4, device=self.device)}
        if want_state:
            out.update(xb0=torch.empty(P, 3, device=self.device), vb0=torch.empty(P, 3, device=self.device),
                       Cb0=torch.empty(P, 3, 3, device=self.device), Fb0=torch.empty(P, 3, 3, device=self.device))
        ob = self._dev(obs_adj)
        mpm.mpm_backward_end(self.ctx, obs_adj=ob, xb0=out.get("xb0"), vb0=out.get("vb0"), Cb0=out.get("Cb0"),
                             Fb0=out.get("Fb0"), pose_grad0=out["pose_grad0"])
        self._keep_e = ob
        return out

    def check_status(self):
        return mpm.mpm_check_status(self.ctx, self.n_envs)

    def tape_length(self):
        return mpm.mpm_tape_length(self.ctx)


def rollout_function():
    """The autograd Function (built lazily so importing this module needs no torch)."""
    torch = _torch()

    class MPMRollout(torch.autograd.Function):
        @staticmethod
        def forward(ctx, batch, group, pose0, actions, x0, v0, C0, F0):
            batch.set_state(x0.detach(), v0.detach(), C0.detach(), F0.detach(), group=group, pose=pose0)
            T = actions.shape[0]
            rewards = torch.stack([batch.step(actions[t].detach(), record=True).clone() for t in range(T)])
            st = batch.get_state()
            ctx.batch = batch
            return rewards, st["x"], st["v"], st["C"], st["F"]

        @staticmethod
        def backward(ctx, g_r, g_x, g_v, g_C, g_F):
            out = ctx.batch.backward(g_x, g_v, g_C, g_F, reward_adj=g_r)
            return None, None, None, out["action_grad"], out["xb0"], out["vb0"], out["Cb0"], out["Fb0"]

    return MPMRollout
