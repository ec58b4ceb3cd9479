"""Host-side pieces of the SAPO update (Sec. 4), on CPU:

- the soft TD(lambda) targets of the recursion equal the explicit weighted average of
  k-step returns that defines them (the TD(lambda) estimate with soft returns);
- the squashed-Gaussian actor's entropy estimate is -log pi(a|o) of the tanh-transformed
  normal, as torch.distributions computes it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2412_12089_gb300 import sapo  # noqa: E402


def test_td_lambda_recursion_equals_definition():
    rng = np.random.default_rng(0)
    H, N, gamma, lam = 6, 3, 0.97, 0.9
    rew = torch.tensor(rng.standard_normal((H, N)))
    soft = torch.tensor(rng.uniform(0, 0.2, (H, N)))
    v_next = torch.tensor(rng.standard_normal((H, N)))  # V(s_1) .. V(s_H)
    got = sapo.td_lambda_targets(rew, soft, v_next, gamma, lam).numpy()
    rt = (rew + soft).numpy()
    V = np.concatenate([np.zeros((1, N)), v_next.numpy()])  # V[t] = V(s_t), t = 1..H

    def G(t, k):  # k-step soft return from t, bootstrapped with V(s_{t+k})
        return sum(gamma ** l * rt[t + l] for l in range(k)) + gamma ** k * V[t + k]

    for t in range(H):
        n = H - t
        want = (1 - lam) * sum(lam ** (l - 1) * G(t, l) for l in range(1, n)) + lam ** (n - 1) * G(t, n)
        assert np.allclose(got[t], want, rtol=1e-12, atol=1e-12), t


def test_actor_entropy_is_negative_log_prob_of_squashed_normal():
    agent = sapo.Agent(obs_dim=7, act_dim=4, cfg=sapo.SapoConfig(hidden=16), device="cpu", seed=1)
    g = torch.Generator().manual_seed(2)
    obs = torch.randn(5, 7, generator=g)
    eps = torch.randn(5, 4, generator=g)
    a, h = agent.act(obs, eps)
    mu, log_std = agent.actor(obs).chunk(2, dim=-1)
    lo, hi = agent.cfg.log_std_range
    log_std = lo + 0.5 * (hi - lo) * (torch.tanh(log_std) + 1.0)
    base = torch.distributions.Normal(mu, log_std.exp())
    dist = torch.distributions.TransformedDistribution(base, [torch.distributions.transforms.TanhTransform()])
    u = mu + log_std.exp() * eps
    assert torch.allclose(a, torch.tanh(u))
    want = -dist.log_prob(torch.tanh(u)).sum(-1)
    # compare away from |a| -> 1, where the transformed density needs atanh(a)
    assert torch.allclose(h, want, rtol=1e-4, atol=1e-4)
    assert torch.all(a.abs() < 1)
