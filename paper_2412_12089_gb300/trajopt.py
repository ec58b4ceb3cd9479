"""First-order trajectory optimisation through the differentiable rollout.

The paper's gradient-based baseline (TrajOpt, Sec. 5) optimises a fixed horizon of actions
directly with AdamW, the gradient of the summed reward flowing back through the simulator.
Here every environment of a batch optimises its own action sequence at once: the forward
rollout records the tape, ``MPMRollout.backward`` runs the library's reverse pass, and the
optimiser updates the actions.  It is the consumer of the action gradients, not part of the
simulator.
"""
from __future__ import annotations

import numpy as np

from .batch import rollout_function


def trajopt(batch, inits, actions0, iters, lr=0.01, betas=(0.7, 0.95), clip=0.5, weight_decay=0.01):
    """Maximise each environment's return sum_t r_t over the horizon len(actions0).

    batch: a Batch with max_steps >= the horizon; inits: per-environment EnvInit;
    actions0: [T, n_envs, A] initial actions.  Returns (actions [T, n_envs, A] as a tensor,
    returns [iters, n_envs] of the iterates, evaluated before each update)."""
    import torch

    MPMRollout = rollout_function()
    dev = batch.device
    x0 = torch.as_tensor(np.concatenate([i.x for i in inits]), device=dev)
    v0 = torch.as_tensor(np.concatenate([i.v for i in inits]), device=dev)
    C0 = torch.as_tensor(np.concatenate([i.C for i in inits]), device=dev)
    F0 = torch.as_tensor(np.concatenate([i.F for i in inits]), device=dev)
    group = torch.as_tensor(np.concatenate([i.group for i in inits]), device=dev)
    pose0 = torch.as_tensor(np.array([s.pose0 for s in batch.specs], np.float32), device=dev)
    a = torch.nn.Parameter(torch.as_tensor(np.asarray(actions0, np.float32), device=dev).clone())
    opt = torch.optim.AdamW([a], lr=lr, betas=betas, weight_decay=weight_decay)
    returns = []
    for _ in range(iters):
        opt.zero_grad()
        rewards = MPMRollout.apply(batch, group, pose0, a, x0, v0, C0, F0)[0]
        ret = rewards.sum(0)
        (-ret.sum()).backward()
        torch.nn.utils.clip_grad_norm_([a], clip)
        opt.step()
        returns.append(ret.detach().cpu().numpy())
    return a.detach(), np.array(returns)
