"""Task observations (App. E tables: subsampled particles x', their mean, actuated pose
components, reach target) of the CUDA path against the FP64 oracle, and the gradient of a
loss on the observations of every recorded state through the reverse pass."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2412_12089_gb300 import workloads as wl

from gpu_helpers import rel_err, split

pytestmark = pytest.mark.gpu


def mixed(T):
    d = wl.dough(n_envs=2, seed=41, n_range=(180, 1500), substeps=4, T=T)  # one env below n_sub = 250
    f = wl.fluid(n_envs=1, seed=42, n=900, substeps=3, T=T)
    specs, inits = d.specs + f.specs, d.inits + f.inits
    A = max(s.action_dim for s in specs)
    acts = np.zeros((T, 3, A), np.float32)
    acts[:, :2, :d.actions.shape[2]] = d.actions[:T]
    acts[:, 2:, :f.actions.shape[2]] = f.actions[:T]
    return wl.Workload("mixed", specs, inits, acts, T)


def to_oracle_layout(row, ns, nsub_max):
    return np.concatenate([row[:3 * ns], row[3 * nsub_max:]])


def test_observation_matches_oracle():
    import torch

    from paper_2412_12089_gb300.batch import Batch

    T = 2
    w = mixed(T)
    b = Batch(w.specs, max_steps=T)
    try:
        b.set_inits(w.inits)
        nss = [min(s.n_sub, s.n_particles) for s in w.specs]
        assert min(nss) < 250 and b.obs_dim == 3 * max(nss) + 10
        obs = [b.observe().cpu().numpy()]
        for t in range(T):
            b.step(torch.as_tensor(w.actions[t]).cuda(), record=True)
            obs.append(b.observe().cpu().numpy())
    finally:
        b.close()
    nsub_max = max(nss)
    for e in range(3):
        s = w.specs[e]
        sp = orc.make_spec(s)
        st = orc.State.from_init(w.inits[e])
        q = np.array(s.pose0, np.float64)
        A = s.action_dim
        for t in range(T + 1):
            ref = orc.observe(sp, st.x, q)
            got = to_oracle_layout(obs[t][e], nss[e], nsub_max)
            tol = 1e-6 if t == 0 else 1e-3
            assert rel_err(got, ref) < tol, (e, t, rel_err(got, ref))
            assert np.all(obs[t][e][3 * nss[e]:3 * nsub_max] == 0.0)
            if t < T:
                st, q, _, _ = orc.rollout(sp, st, q, w.actions[t:t + 1, e, :A].astype(np.float64))


def test_observation_gradients_match_oracle():
    import torch

    from paper_2412_12089_gb300.batch import Batch

    T = 2
    w = mixed(T)
    rng = np.random.default_rng(43)
    b = Batch(w.specs, max_steps=T)
    try:
        b.set_inits(w.inits)
        for t in range(T):
            b.step(torch.as_tensor(w.actions[t]).cuda(), record=True)
        cw = rng.standard_normal((T + 1, 3, b.obs_dim)).astype(np.float32)
        g = b.backward(obs_adj=cw)
        g = {k: v.cpu().numpy() for k, v in g.items()}
        # consumed: a second backward without observation adjoints sees none
        b.set_inits(w.inits)
        for t in range(T):
            b.step(torch.as_tensor(w.actions[t]).cuda(), record=True)
        g0 = b.backward(reward_adj=np.zeros((T, 3), np.float32))
        assert float(g0["action_grad"].abs().max()) == 0.0
        nsub_max = (b.obs_dim - 10) // 3
    finally:
        b.close()
    for e in range(3):
        s = w.specs[e]
        sp = orc.make_spec(s)
        so = orc.State.from_init(w.inits[e])
        ns = min(s.n_sub, s.n_particles)
        A = s.action_dim
        oa = np.stack([to_oracle_layout(cw[t, e].astype(np.float64), ns, nsub_max) for t in range(T + 1)])
        ag, (xb, vb, Cb, Fb), qb = orc.rollout_adj(sp, so, np.array(s.pose0, np.float64),
                                                   w.actions[:T, e, :A].astype(np.float64), obs_adj=oa)
        assert rel_err(g["action_grad"][:, e, :A], ag) < 1e-3, (e, rel_err(g["action_grad"][:, e, :A], ag))
        assert rel_err(split(w, g["xb0"])[e], xb) < 1e-3, (e, "xb0")
        assert rel_err(g["pose_grad0"][e], qb) < 1e-3, (e, g["pose_grad0"][e], qb)
