"""Maximum-entropy first-order actor-critic update (SAPO, Sec. 4 and App. B) on the batched
simulator: a closed-loop consumer of the step-wise reverse pass.

One iteration starts from the batch's current state:

1. Rollout.  H control steps with the stochastic actor a_t = tanh(mu + sigma eps) on the
   observations o_t (the App. E layout of ``mpm_observe``), recorded on the tape.
2. Actor.  Per environment, maximise the entropy-augmented H-step return plus the discounted
   soft value of the last state (Sec. 4.1's first-order estimate):
       J = sum_t gamma^t (r_t + alpha h_hat_t) + gamma^H mean_i V_i(o_H),
   where h_hat_t = (h_t + |H_bar|) / (2 |H_bar|) is the normalised entropy estimate (design
   choice II), and J is averaged over environments.  Its gradient goes back through the
   simulator one step at a time: ``backward_step`` gives the adjoint of a_t, which goes
   through the actor to o_t, and the adjoint of o_t enters the reverse of step t - 1.
3. Temperature.  One step on alpha (h - H_bar) with the unnormalised entropy (design
   choice I).
4. Critics.  TD(lambda) targets from soft k-step returns with the minimum over the two
   critics (design choice IV), then K mini-epochs of mean-squared regression.

The hyperparameters follow the paper's table for SAPO: gamma 0.99, lambda 0.95, actor lr
2e-3, critic lr 5e-4, entropy lr 5e-3, Adam betas (0.7, 0.95), gradient clip 0.5, log sigma
in [-5, 2], two critics, LayerNorm + SiLU MLPs, target entropy -dim(A)/2, initial
temperature 1.  The point-cloud encoder is replaced by the flat observation vector.  The
actor and critics are small torch modules; every simulation step and its reverse run in the
library.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

from . import mpm


def _torch():
    import torch

    return torch


@dataclass
class SapoConfig:
    horizon: int = 32
    gamma: float = 0.99
    lam: float = 0.95
    actor_lr: float = 2e-3
    critic_lr: float = 5e-4
    alpha_lr: float = 5e-3
    betas: tuple = (0.7, 0.95)
    grad_clip: float = 0.5
    critic_epochs: int = 16
    hidden: int = 128
    log_std_range: tuple = (-5.0, 2.0)
    init_alpha: float = 1.0


def _mlp(n_in, n_out, hidden):
    nn = _torch().nn
    return nn.Sequential(nn.Linear(n_in, hidden), nn.LayerNorm(hidden), nn.SiLU(),
                         nn.Linear(hidden, hidden), nn.LayerNorm(hidden), nn.SiLU(), nn.Linear(hidden, n_out))


class Agent:
    """Squashed-Gaussian actor with state-dependent variance (design choice III), two critics
    and the entropy temperature."""

    def __init__(self, obs_dim, act_dim, cfg: SapoConfig = SapoConfig(), device="cuda", seed=0):
        torch = _torch()
        torch.manual_seed(seed)
        self.cfg = cfg
        self.act_dim = act_dim
        self.actor = _mlp(obs_dim, 2 * act_dim, cfg.hidden).to(device)
        self.critics = [_mlp(obs_dim, 1, cfg.hidden).to(device) for _ in range(2)]
        self.log_alpha = torch.tensor(math.log(cfg.init_alpha), device=device, requires_grad=True)
        self.target_entropy = -act_dim / 2.0
        self.opt_actor = torch.optim.Adam(self.actor.parameters(), lr=cfg.actor_lr, betas=cfg.betas)
        self.opt_critic = torch.optim.Adam([p for c in self.critics for p in c.parameters()], lr=cfg.critic_lr,
                                           betas=cfg.betas)
        self.opt_alpha = torch.optim.Adam([self.log_alpha], lr=cfg.alpha_lr, betas=cfg.betas)

    @property
    def alpha(self):
        return self.log_alpha.exp()

    def act(self, obs, eps):
        """Reparameterised action a = tanh(mu + sigma eps) and its entropy estimate
        h = -log pi(a | o) (one sample, with the tanh change of variables)."""
        torch = _torch()
        mu, log_std = self.actor(obs).chunk(2, dim=-1)
        lo, hi = self.cfg.log_std_range
        log_std = lo + 0.5 * (hi - lo) * (torch.tanh(log_std) + 1.0)
        u = mu + log_std.exp() * eps
        a = torch.tanh(u)
        # log N(u; mu, sigma) - log(1 - tanh(u)^2), the latter as 2 (log 2 - u - softplus(-2u))
        logp = (-0.5 * eps * eps - log_std - 0.5 * math.log(2.0 * math.pi)).sum(-1)
        logp = logp - (2.0 * (math.log(2.0) - u - torch.nn.functional.softplus(-2.0 * u))).sum(-1)
        return a, -logp

    def value(self, obs, reduce="mean"):
        torch = _torch()
        v = torch.stack([c(obs).squeeze(-1) for c in self.critics])
        return v.mean(0) if reduce == "mean" else v.min(0).values

    def h_hat(self, h):
        H = abs(self.target_entropy)
        return (h + H) / (2.0 * H)


def _check_batch(batch, agent):
    if batch.A < agent.act_dim:
        raise ValueError(f"the batch takes {batch.A} action entries, the actor gives {agent.act_dim}")
    if batch.max_steps < agent.cfg.horizon:
        raise ValueError("the batch's tape must hold the horizon (max_steps >= horizon)")


def _pad(a, A):
    torch = _torch()
    if a.shape[1] == A:
        return a
    return torch.cat([a, a.new_zeros(a.shape[0], A - a.shape[1])], dim=1)


def objective(batch, agent, eps, horizon=None):
    """J averaged over environments for fixed noise eps [H, n_envs, act_dim], forward only
    (not recorded), from the batch's current state.  The state is left at step H."""
    torch = _torch()
    cfg = agent.cfg
    H = horizon or cfg.horizon
    N = batch.n_envs
    J = torch.zeros(N, device=batch.device)
    with torch.no_grad():
        alpha = agent.alpha
        for t in range(H):
            o = batch.observe()
            a, h = agent.act(o, eps[t])
            r = batch.step(_pad(a, batch.A)).clone()
            J += cfg.gamma ** t * (r + alpha * agent.h_hat(h))
        J += cfg.gamma ** H * agent.value(batch.observe())
    return float(J.mean())


def actor_gradient(batch, agent, eps, horizon=None):
    """Rollout with noise eps [H, n_envs, act_dim] from the batch's current state, recorded,
    then the closed-loop gradient of -J into the actor's .grad (zeroed first).  Returns the
    rollout's buffer: observations [H + 1, N, obs_dim], rewards and entropies [H, N]."""
    torch = _torch()
    cfg = agent.cfg
    H = horizon or cfg.horizon
    _check_batch(batch, agent)
    N = batch.n_envs
    mpm.mpm_reset_tape(batch.ctx)
    obs, acts, ents, rews = [], [], [], []
    alpha = agent.alpha.detach()
    for t in range(H):
        o = batch.observe().detach().requires_grad_(True)
        a, h = agent.act(o, eps[t])
        r = batch.step(_pad(a.detach(), batch.A), record=True).clone()
        obs.append(o)
        acts.append(a)
        ents.append(h)
        rews.append(r)
    oH = batch.observe().detach().requires_grad_(True)
    for p in agent.actor.parameters():
        p.grad = None
    # loss = -J / N: the terminal value's adjoint on o_H goes into the last reverse step
    lossH = -(cfg.gamma ** H / N) * agent.value(oH).sum()
    og = torch.autograd.grad(lossH, oH)[0]
    batch.backward_begin()
    params = list(agent.actor.parameters())
    for t in range(H - 1, -1, -1):
        rb = torch.full((N,), -(cfg.gamma ** t) / N, device=batch.device)
        ts, ag = batch.backward_step(reward_adj=rb, obs_adj=og)
        assert ts == t
        # step t's local graph: the action (its total adjoint from the simulator) and the
        # entropy term, both functions of o_t and the actor's parameters
        local = (acts[t] * ag[:, :agent.act_dim]).sum() - (cfg.gamma ** t / N) * (alpha * agent.h_hat(ents[t])).sum()
        grads = torch.autograd.grad(local, params + [obs[t]], allow_unused=True)
        for p, g in zip(params, grads[:-1]):
            if g is not None:
                p.grad = g if p.grad is None else p.grad + g
        og = grads[-1]
    batch.backward_end(obs_adj=og)
    return {"obs": torch.stack([o.detach() for o in obs] + [oH.detach()]), "rew": torch.stack(rews),
            "ent": torch.stack([h.detach() for h in ents])}


def td_lambda_targets(rew, soft, v_next, gamma, lam):
    """Soft TD(lambda) targets over the window: G_t = r~_t + gamma ((1 - lambda) v_{t+1} +
    lambda G_{t+1}), G_{H-1} = r~_{H-1} + gamma v_H, with r~ = r + alpha h_hat.
    rew, soft: [H, N]; v_next: [H, N] values of o_1..o_H."""
    torch = _torch()
    H = rew.shape[0]
    G = torch.empty_like(rew)
    nxt = v_next[H - 1]
    for t in range(H - 1, -1, -1):
        rt = rew[t] + soft[t]
        if t == H - 1:
            G[t] = rt + gamma * v_next[t]
        else:
            G[t] = rt + gamma * ((1.0 - lam) * v_next[t] + lam * nxt)
        nxt = G[t]
    return G


def iteration(batch, agent, eps):
    """One SAPO update (actor, temperature, critics) from the batch's current state; the
    state then is at step H.  Returns statistics of the iteration."""
    torch = _torch()
    cfg = agent.cfg
    buf = actor_gradient(batch, agent, eps)
    torch.nn.utils.clip_grad_norm_(agent.actor.parameters(), cfg.grad_clip)
    agent.opt_actor.step()
    # temperature: alpha (h - H_bar) with the unnormalised entropy
    h = buf["ent"]
    agent.opt_alpha.zero_grad()
    (agent.alpha * (h.mean() - agent.target_entropy)).backward()
    agent.opt_alpha.step()
    # critics on soft TD(lambda) targets with the minimum of the two critics
    with torch.no_grad():
        alpha = agent.alpha
        soft = alpha * agent.h_hat(h)
        v_next = agent.value(buf["obs"][1:], reduce="min")
        target = td_lambda_targets(buf["rew"], soft, v_next, cfg.gamma, cfg.lam)
    o = buf["obs"][:-1].reshape(-1, buf["obs"].shape[-1])
    y = target.reshape(-1)
    losses = []
    for _ in range(cfg.critic_epochs):
        agent.opt_critic.zero_grad()
        loss = sum(((c(o).squeeze(-1) - y) ** 2).mean() for c in agent.critics)
        loss.backward()
        agent.opt_critic.step()
        losses.append(float(loss.detach()))
    return {"reward": float(buf["rew"].mean()), "entropy": float(h.mean()), "alpha": float(agent.alpha.detach()),
            "critic_loss_first": losses[0], "critic_loss_last": losses[-1]}
