"""Step-wise reverse pass and its closed-loop consumer (SAPO actor update).

- Reversing one recorded step at a time, with the same reward and observation adjoints,
  gives the whole-tape backward's action, initial-state and pose gradients.
- The closed-loop actor gradient (the adjoint of a_t through the policy into o_t, and on into
  the reverse of step t - 1) matches central differences of the objective J computed by
  forward-only rollouts with the same noise.
- SAPO iterations run end to end and move the temperature and the critics.
"""
import numpy as np
import pytest

from paper_2412_12089_gb300 import workloads as wl

from gpu_helpers import rel_err

pytestmark = pytest.mark.gpu


def test_stepwise_equals_whole_tape():
    import torch

    from paper_2412_12089_gb300.batch import Batch

    T = 3
    w = wl.fluid(n_envs=3, seed=61, n=1200, substeps=4, T=T)
    rng = np.random.default_rng(61)
    b = Batch(w.specs, max_steps=T)
    try:
        b.set_inits(w.inits)
        for t in range(T):
            b.step(torch.as_tensor(w.actions[t]).cuda(), record=True)
        N, D = b.n_envs, b.obs_dim
        rbar = rng.standard_normal((T, N)).astype(np.float32)
        oa = rng.standard_normal((T + 1, N, D)).astype(np.float32)
        ref = {k: v.cpu().numpy() for k, v in b.backward(reward_adj=rbar, obs_adj=oa).items()}
        b.backward_begin()
        with pytest.raises(Exception):
            b.backward(reward_adj=rbar)  # refused while a step-wise pass is open
        ag = np.zeros((T, N, b.A), np.float32)
        with pytest.raises(Exception):
            b.backward_end()  # steps left
        for t in range(T - 1, -1, -1):
            ts, g = b.backward_step(reward_adj=rbar[t], obs_adj=oa[t + 1])
            assert ts == t
            ag[t] = g.cpu().numpy()
        with pytest.raises(Exception):
            b.backward_step()  # every step reversed
        got = {k: v.cpu().numpy() for k, v in b.backward_end(obs_adj=oa[0], want_state=True).items()}
    finally:
        b.close()
    assert rel_err(ag, ref["action_grad"]) < 1e-4, rel_err(ag, ref["action_grad"])
    for k in ("xb0", "vb0", "Fb0", "pose_grad0"):
        assert rel_err(got[k], ref[k]) < 1e-4, (k, rel_err(got[k], ref[k]))


@pytest.mark.parametrize("task", ["fluid", "softjumper"])
def test_closed_loop_gradient_matches_finite_differences(task):
    import torch

    from paper_2412_12089_gb300 import sapo
    from paper_2412_12089_gb300.batch import Batch

    H = 3
    if task == "fluid":
        w = wl.fluid(n_envs=2, seed=62, n=1500, substeps=5, T=H)
    else:  # tetrahedral FEM: observations of the mesh vertices, 220 activations
        w = wl.softjumper(n_envs=2, seed=62, T=H)
    A = w.specs[0].action_dim
    b = Batch(w.specs, max_steps=H)
    try:
        agent = sapo.Agent(b.obs_dim, A, sapo.SapoConfig(horizon=H, hidden=32), device=b.device, seed=3)
        gen = torch.Generator(device="cpu").manual_seed(5)
        eps = torch.randn(H, b.n_envs, A, generator=gen).to(b.device)
        b.set_inits(w.inits)
        sapo.actor_gradient(b, agent, eps)
        params = list(agent.actor.parameters())
        g = torch.cat([p.grad.reshape(-1) for p in params])  # gradient of -J
        d = -g / g.norm()
        theta = [p.detach().clone() for p in params]
        gd = float(-(g * d).sum())  # dJ along d
        J0 = None
        for h in (3e-3, 1e-3):
            vals = []
            for sgn in (1.0, -1.0):
                off = 0
                with torch.no_grad():
                    for p, t0 in zip(params, theta):
                        n = p.numel()
                        p.copy_(t0 + sgn * h * d[off:off + n].reshape(p.shape))
                        off += n
                b.set_inits(w.inits)
                vals.append(sapo.objective(b, agent, eps))
            fd = (vals[0] - vals[1]) / (2 * h)
            J0 = vals
            assert abs(fd - gd) <= 3e-2 * abs(gd), (h, fd, gd, J0)
    finally:
        b.close()


def test_sapo_iterations_run():
    import torch

    from paper_2412_12089_gb300 import sapo
    from paper_2412_12089_gb300.batch import Batch

    H = 4
    w = wl.fluid(n_envs=4, seed=63, n=1500, substeps=5, T=H)
    b = Batch(w.specs, max_steps=H)
    try:
        agent = sapo.Agent(b.obs_dim, 3, sapo.SapoConfig(horizon=H, hidden=64), device=b.device, seed=4)
        gen = torch.Generator(device="cpu").manual_seed(6)
        alpha0 = float(agent.alpha.detach())
        stats = []
        for it in range(3):
            b.set_inits(w.inits)
            eps = torch.randn(H, b.n_envs, 3, generator=gen).to(b.device)
            stats.append(sapo.iteration(b, agent, eps))
        code, flags = b.check_status()
    finally:
        b.close()
    assert code == 0 and not flags.any()
    for s in stats:
        assert all(np.isfinite(v) for v in s.values()), s
        assert s["critic_loss_last"] < s["critic_loss_first"], s
    assert float(agent.alpha.detach()) != alpha0
