"""Kept substep states (mpm_options.keep_fraction): the recorded forward pass writes each
control step's substep states to slot (t mod n) of a keep buffer, and the reverse pass of the
last n recorded steps reads them instead of recomputing them from the step's checkpoint
(Sec. 4.1 recomputes; keeping them is a trade of memory for time).  Both reverse paths must
give the same result: every test runs a horizon with nothing kept, part kept and all kept,
and checks the gradients against each other and against the FP64 oracle."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2412_12089_gb300 import workloads as wl

from gpu_helpers import rel_err, split

pytestmark = pytest.mark.gpu


def _run(w, T, monkeypatch, keep, stepwise=False):
    """Record T steps and reverse them with reward adjoints 1.  keep: None (the default
    share of memory), 0 (keep_fraction < 0: nothing kept) or a cap on the kept steps."""
    import torch

    from paper_2412_12089_gb300 import mpm
    from paper_2412_12089_gb300.batch import Batch

    if keep is None or keep == 0:
        monkeypatch.delenv("MPM_KEEP_STEPS", raising=False)
    else:
        monkeypatch.setenv("MPM_KEEP_STEPS", str(keep))
    b = Batch(w.specs, max_steps=T, keep_fraction=-1.0 if keep == 0 else 0.0)
    kept = mpm.mpm_kept_steps(b.ctx)
    b.set_inits(w.inits)
    rews = [b.step(torch.as_tensor(w.actions[t]).cuda(), record=True).clone() for t in range(T)]
    xT = b.get_state()["x"].cpu().numpy()
    rbar = torch.ones(T, w.n_envs, device="cuda")
    if stepwise:
        b.backward_begin()
        ag = np.zeros((T, w.n_envs, b.A), np.float32)
        for t in range(T - 1, -1, -1):
            step, g_t = b.backward_step(reward_adj=rbar[t])
            ag[step] = g_t.cpu().numpy()
        out = {k: v.cpu().numpy() for k, v in b.backward_end(want_state=True).items()}
        out["action_grad"] = ag
    else:
        out = {k: v.cpu().numpy() for k, v in b.backward(reward_adj=rbar).items()}
    torch.cuda.synchronize()
    b.close()
    return kept, torch.stack(rews).cpu().numpy(), xT, out


def _oracle_grads(w, T, e):
    s = w.specs[e]
    sp = orc.make_spec(s)
    so = orc.State.from_init(w.inits[e])
    A = s.action_dim
    ag, (xb, vb, Cb, Fb), _ = orc.rollout_adj(sp, so, np.array(s.pose0, np.float64),
                                              w.actions[:T, e, :A].astype(np.float64), rbar=np.ones(T))
    return ag, xb, vb


@pytest.mark.parametrize("name", ["fluid", "dough"])
def test_kept_and_recomputed_reverse_agree(name, monkeypatch):
    """Four recorded steps of four substeps: nothing kept (every step recomputed), the last
    two kept, all kept.  Forward results and gradients agree across the three (they differ
    only by the order of P2G's float atomics), and match the oracle."""
    T, S = 4, 4
    if name == "fluid":
        w = wl.fluid(n_envs=2, seed=31, n=1200, substeps=S, T=T)
    else:
        w = wl.dough(n_envs=2, seed=32, n_range=(600, 2000), substeps=S, T=T)
    runs = {k: _run(w, T, monkeypatch, k) for k in (0, 2, None)}
    assert runs[0][0] == 0 and runs[2][0] == 2 and runs[None][0] == T
    _, rew0, x0, g0 = runs[0]
    for k in (2, None):
        _, rew, x, g = runs[k]
        assert rel_err(x, x0) < 1e-5, (k, rel_err(x, x0))
        assert rel_err(rew, rew0) < 1e-4, (k, rel_err(rew, rew0))
        for q in ("action_grad", "xb0", "vb0", "Cb0", "Fb0"):
            assert rel_err(g[q], g0[q]) < 1e-4, (k, q, rel_err(g[q], g0[q]))
    g = runs[2][3]
    for e in range(w.n_envs):
        ag, xb, vb = _oracle_grads(w, T, e)
        A = w.specs[e].action_dim
        assert rel_err(g["action_grad"][:, e, :A], ag) < 1e-3, (e, rel_err(g["action_grad"][:, e, :A], ag))
        assert rel_err(split(w, g["xb0"])[e], xb) < 1e-3, e
        assert rel_err(split(w, g["vb0"])[e], vb) < 1e-3, e


def test_mixed_substep_counts_partly_kept(monkeypatch):
    """Environments of two materials with 5 and 3 substeps in one batch, three recorded steps
    with the last one kept: each environment's gradients match its oracle."""
    T = 3
    d = wl.dough(n_envs=2, seed=33, n_range=(500, 2000), substeps=5, T=T)
    f = wl.fluid(n_envs=1, seed=34, n=1000, substeps=3, T=T)
    specs, inits = d.specs + f.specs, d.inits + f.inits
    A = max(s.action_dim for s in specs)
    acts = np.zeros((T, 3, A), np.float32)
    acts[:, :2, :d.actions.shape[2]] = d.actions[:T]
    acts[:, 2:, :f.actions.shape[2]] = f.actions[:T]
    w = wl.Workload("mixed", specs, inits, acts, T)
    kept, _, _, g = _run(w, T, monkeypatch, 1)
    assert kept == 1
    for e in range(3):
        ag, xb, vb = _oracle_grads(w, T, e)
        Ae = w.specs[e].action_dim
        assert rel_err(g["action_grad"][:, e, :Ae], ag) < 1e-3, (e, rel_err(g["action_grad"][:, e, :Ae], ag))
        assert rel_err(split(w, g["xb0"])[e], xb) < 1e-3, (e, "xb0")
        assert rel_err(split(w, g["vb0"])[e], vb) < 1e-3, (e, "vb0")


def test_stepwise_reverse_over_kept_and_recomputed_steps(monkeypatch):
    """The step-wise reverse pass (mpm_backward_begin / _step / _end) over four recorded
    steps, the last two kept, equals the whole-tape reverse pass."""
    T = 4
    w = wl.fluid(n_envs=2, seed=35, n=1000, substeps=3, T=T)
    kept, _, _, g_whole = _run(w, T, monkeypatch, 2)
    kept2, _, _, g_step = _run(w, T, monkeypatch, 2, stepwise=True)
    assert kept == kept2 == 2
    for q in ("action_grad", "xb0", "vb0", "Cb0", "Fb0"):
        assert rel_err(g_step[q], g_whole[q]) < 1e-4, (q, rel_err(g_step[q], g_whole[q]))
