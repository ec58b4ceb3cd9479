"""The action gradients are usable: AdamW trajectory optimisation through the differentiable
rollout raises the return of every environment of a batch (fluid container reaching a
target), and the autograd path's gradient equals the explicit reverse pass's."""
import numpy as np
import pytest

from paper_2412_12089_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_trajopt_raises_returns():
    from paper_2412_12089_gb300.batch import Batch
    from paper_2412_12089_gb300.trajopt import trajopt

    T = 4
    w = wl.fluid(n_envs=4, seed=21, n=1500, substeps=5, T=T)
    b = Batch(w.specs, max_steps=T)
    try:
        _, R = trajopt(b, w.inits, w.actions[:T], iters=12, lr=0.3)
    finally:
        b.close()
    assert np.all(np.isfinite(R))
    gain = R[-1] - R[0]
    assert gain.mean() > 0 and np.count_nonzero(gain > 0) >= 3, (R[0], R[-1])


def test_autograd_gradient_equals_explicit_backward():
    import torch

    from paper_2412_12089_gb300.batch import Batch, rollout_function

    T = 2
    w = wl.dough(n_envs=2, seed=22, n_range=(800, 1500), substeps=4, T=T)
    b = Batch(w.specs, max_steps=T)
    try:
        b.set_inits(w.inits)
        for t in range(T):
            b.step(torch.as_tensor(w.actions[t]).cuda(), record=True)
        ref = b.backward(reward_adj=np.ones((T, 2), np.float32))["action_grad"].clone()
        dev = b.device
        x0 = torch.as_tensor(np.concatenate([i.x for i in w.inits]), device=dev)
        v0 = torch.as_tensor(np.concatenate([i.v for i in w.inits]), device=dev)
        C0 = torch.as_tensor(np.concatenate([i.C for i in w.inits]), device=dev)
        F0 = torch.as_tensor(np.concatenate([i.F for i in w.inits]), device=dev)
        g = torch.as_tensor(np.concatenate([i.group for i in w.inits]), device=dev)
        pose0 = torch.as_tensor(np.array([s.pose0 for s in w.specs], np.float32), device=dev)
        a = torch.as_tensor(w.actions[:T], device=dev).clone().requires_grad_(True)
        rewards = rollout_function().apply(b, g, pose0, a, x0, v0, C0, F0)[0]
        rewards.sum().backward()
        got = a.grad
    finally:
        b.close()
    err = (got - ref).abs().max().item() / max(ref.abs().max().item(), 1e-12)
    assert err < 1e-5, err
