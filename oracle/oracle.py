"""ctypes binding of the FP64 CPU oracle (mpm_oracle.c).

TEST INFRASTRUCTURE ONLY.  Imported by tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; never by the product package.  The oracle is a plain,
single-threaded FP64 implementation of arXiv 2412.12089 App. D.3 (MLS-MPM with the von
Mises / fluid / neo-Hookean laws and softened SDF contact) and of its exact discrete
adjoint (Sec. 4.1).

Every function takes numpy arrays in particle-major layout: x (n,3), v (n,3),
C (n,3,3), F (n,3,3), group (n,) int32; they are converted to FP64 here.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmpm_oracle.so")
SRC = os.path.join(HERE, "mpm_oracle.c")

MAT = {"neohookean": 0, "vonmises": 1, "fluid": 2, "muscle": 3}
COLL = {"none": 0, "capsule": 1, "box": 2, "container": 3, "capsules": 4}
REWARD = {"none": 0, "flat": 1, "reach": 2, "jump": 3}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so the FP32 binning mirror rounds
    each operation separately)."""
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "mpm_oracle.h"))
    ):
        tmp = LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-shared",
                               "-fPIC", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


class OrcSpec(ct.Structure):
    _fields_ = [
        ("G", ct.c_int), ("S", ct.c_int), ("bound", ct.c_int), ("material", ct.c_int),
        ("coll_kind", ct.c_int), ("n_coll_act", ct.c_int), ("act_map", ct.c_int * 4),
        ("n_groups", ct.c_int), ("reward_kind", ct.c_int), ("n_sub", ct.c_int),
        ("dt", ct.c_double), ("gravity", ct.c_double * 3), ("p_mass", ct.c_double),
        ("p_vol", ct.c_double), ("mu", ct.c_double), ("lam", ct.c_double),
        ("yield_stress", ct.c_double), ("c_y", ct.c_double), ("bulk", ct.c_double),
        ("visc", ct.c_double), ("act_stress", ct.c_double), ("coll_dims", ct.c_double * 4),
        ("coll_mu", ct.c_double), ("alpha", ct.c_double), ("act_scale", ct.c_double * 4),
        ("ground_mu", ct.c_double), ("rparam", ct.c_double * 4), ("n_caps", ct.c_int),
        ("cap_offset", ct.c_double * 3),
    ]


_lib = None
_D = ct.POINTER(ct.c_double)
_I = ct.POINTER(ct.c_int)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ct.CDLL(LIB_PATH)
        P = ct.POINTER(OrcSpec)
        L.orc_svd3.argtypes = [_D, _D, _D, _D]
        L.orc_tau.argtypes = [P, _D, _D, ct.c_double, _D]
        L.orc_tau_vjp.argtypes = [P, _D, _D, ct.c_double, _D, _D, _D, _D]
        L.orc_project.argtypes = [P, _D, _D]
        L.orc_project_vjp.argtypes = [P, _D, _D, _D]
        L.orc_collider.argtypes = [P, _D, _D, _D, _D, _D, _D, _D]
        L.orc_weights.argtypes = [ct.c_double, _D, _D]
        L.orc_p2g.argtypes = [P, ct.c_int, _D, _D, _D, _D, _I, _D, _D]
        L.orc_p2g.restype = ct.c_int
        L.orc_grid_update.argtypes = [P, _D, _D, _D, _D]
        L.orc_g2p.argtypes = [P, ct.c_int, _D, _D, _D, _D, _D]
        L.orc_g2p.restype = ct.c_int
        L.orc_substep.argtypes = [P, ct.c_int, _D, _D, _D, _D, _I, _D, _D, _D]
        L.orc_substep.restype = ct.c_int
        L.orc_substep_adj.argtypes = [P, ct.c_int, _D, _D, _D, _D, _I, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D]
        L.orc_substep_adj.restype = ct.c_int
        L.orc_reward.argtypes = [P, ct.c_int, _D, _D, _D, _D]
        L.orc_reward.restype = ct.c_double
        L.orc_reward_adj.argtypes = [P, ct.c_int, _D, _D, _D, _D, ct.c_double, _D, _D, _D, _D]
        L.orc_rollout.argtypes = [P, ct.c_int, _D, _D, _D, _D, _I, _D, _D, ct.c_int, _D]
        L.orc_rollout.restype = ct.c_int
        L.orc_rollout_adj.argtypes = [P, ct.c_int, _D, _D, _D, _D, _I, _D, _D, ct.c_int, _D, _D, _D, _D, _D,
                                      _D, _D, _D, _D, _D, _D]
        L.orc_rollout_adj.restype = ct.c_int
        L.orc_rollout_adj_obs.argtypes = [P, ct.c_int, _D, _D, _D, _D, _I, _D, _D, ct.c_int, _D, _D, _D, _D, _D,
                                          _D, _D, _D, _D, _D, _D, _D]
        L.orc_rollout_adj_obs.restype = ct.c_int
        L.orc_obs_dim.argtypes = [P, ct.c_int]
        L.orc_obs_dim.restype = ct.c_int
        L.orc_observe.argtypes = [P, ct.c_int, _D, _D, _D]
        L.orc_bin_keys_f32.argtypes = [ct.c_int, ct.POINTER(ct.c_float), ct.c_int, ct.POINTER(ct.c_uint)]
        L.orc_stable_sort_u32.argtypes = [ct.c_int, ct.POINTER(ct.c_uint), ct.POINTER(ct.c_uint)]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _arr(a, shape=None):
    out = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        out = out.reshape(shape)
    return out


def lame(E, nu):
    return E / (2.0 * (1.0 + nu)), E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))


def make_spec(es) -> OrcSpec:
    """OrcSpec from a workloads.EnvSpec (or anything with the same attributes)."""
    s = OrcSpec()
    s.G, s.S, s.bound = es.grid_res, es.substeps, es.bound
    s.material = MAT[es.material]
    s.coll_kind = COLL[es.collider]
    s.n_coll_act = 4 * es.n_caps if es.collider == "capsules" else len(es.act_map)
    s.n_caps = es.n_caps if es.collider == "capsules" else 0
    for i in range(3):
        s.cap_offset[i] = es.cap_offset[i]
    for j in range(4):
        s.act_map[j] = es.act_map[j] if j < len(es.act_map) else 0
        s.act_scale[j] = es.act_scale[j] if j < len(es.act_scale) else 0.0
        s.coll_dims[j] = es.coll_dims[j]
        s.rparam[j] = es.rparam[j]
    s.n_groups = es.n_groups
    s.reward_kind = REWARD[es.reward]
    s.n_sub = es.n_sub
    s.dt = es.dt
    for i in range(3):
        s.gravity[i] = es.gravity[i]
    s.p_vol = es.p_vol
    s.p_mass = es.rho * es.p_vol
    if es.material in ("neohookean", "vonmises", "muscle"):
        s.mu, s.lam = lame(es.E, es.nu)
    s.yield_stress, s.c_y = es.yield_stress, es.c_y
    s.bulk, s.visc, s.act_stress = es.bulk, es.visc, es.act_stress
    s.coll_mu, s.alpha, s.ground_mu = es.coll_mu, es.alpha, es.ground_mu
    return s


def pose_len(spec):
    """Entries of the pose vector: 4, or 4 per capsule for the multi-capsule collider."""
    return 4 * spec.n_caps if spec.coll_kind == COLL["capsules"] else 4


def initial_pose(es):
    """Initial pose vector of an EnvSpec: pose0, or for the multi-capsule collider capsule j
    at pose0 + j * cap_offset (same angle)."""
    p0 = np.asarray(es.pose0, np.float64)
    if es.collider != "capsules":
        return p0.copy()
    return np.concatenate([p0 + np.array([*(j * np.asarray(es.cap_offset, np.float64)), 0.0])
                           for j in range(es.n_caps)])


class State:
    """FP64 particle state (particle-major)."""

    def __init__(self, x, v, C, F, group=None):
        n = np.asarray(x).shape[0]
        self.x = _arr(x, (n, 3)).copy()
        self.v = _arr(v, (n, 3)).copy()
        self.C = _arr(C, (n, 3, 3)).copy()
        self.F = _arr(F, (n, 3, 3)).copy()
        g = np.full(n, -1, np.int32) if group is None else np.asarray(group, np.int32)
        self.group = np.ascontiguousarray(g)

    @classmethod
    def from_init(cls, init):
        return cls(init.x, init.v, init.C, init.F, init.group)

    @property
    def n(self):
        return self.x.shape[0]

    def copy(self):
        return State(self.x, self.v, self.C, self.F, self.group)

    def arrays(self):
        return self.x, self.v, self.C, self.F


def _gp(g):
    return g.ctypes.data_as(_I)


# ------------------------------------------------------------------------ building blocks

def svd3(F):
    F = _arr(F, (3, 3))
    U, s, V = np.zeros((3, 3)), np.zeros(3), np.zeros((3, 3))
    lib().orc_svd3(_d(F), _d(U), _d(s), _d(V))
    return U, s, V


def tau(spec, F, C=None, a_g=0.0):
    F = _arr(F, (3, 3))
    C = np.zeros((3, 3)) if C is None else _arr(C, (3, 3))
    out = np.zeros((3, 3))
    lib().orc_tau(ct.byref(spec), _d(F), _d(C), a_g, _d(out))
    return out


def tau_vjp(spec, F, C, a_g, taub):
    F, C, taub = _arr(F, (3, 3)), _arr(C, (3, 3)), _arr(taub, (3, 3))
    Fb, Cb, ab = np.zeros((3, 3)), np.zeros((3, 3)), np.zeros(1)
    lib().orc_tau_vjp(ct.byref(spec), _d(F), _d(C), a_g, _d(taub), _d(Fb), _d(Cb), _d(ab))
    return Fb, Cb, ab[0]


def project(spec, Ft):
    Ft = _arr(Ft, (3, 3))
    out = np.zeros((3, 3))
    lib().orc_project(ct.byref(spec), _d(Ft), _d(out))
    return out


def project_vjp(spec, Ft, Fob):
    Ft, Fob = _arr(Ft, (3, 3)), _arr(Fob, (3, 3))
    out = np.zeros((3, 3))
    lib().orc_project_vjp(ct.byref(spec), _d(Ft), _d(Fob), _d(out))
    return out


def collider(spec, xw, q, u=None):
    pl = pose_len(spec)
    xw, q = _arr(xw, (3,)), _arr(q, (pl,))
    u = np.zeros(pl) if u is None else _arr(u, (pl,))
    d, n, H, vb = np.zeros(1), np.zeros(3), np.zeros((3, 3)), np.zeros(3)
    lib().orc_collider(ct.byref(spec), _d(xw), _d(q), _d(u), _d(d), _d(n), _d(H), _d(vb))
    return d[0], n, H, vb


def weights(fx):
    w, dw = np.zeros(3), np.zeros(3)
    lib().orc_weights(float(fx), _d(w), _d(dw))
    return w, dw


def p2g(spec, st: State, act=None):
    G = spec.G
    g = np.zeros((G, G, G, 4))  # index [iz, iy, ix]
    a = _arr(np.zeros(1) if act is None else act)
    status = lib().orc_p2g(ct.byref(spec), st.n, _d(st.x), _d(st.v), _d(st.C), _d(st.F), _gp(st.group), _d(a), _d(g))
    return g, status


def grid_update(spec, g, q=None, u=None):
    G = spec.G
    pl = pose_len(spec)
    g = _arr(g, (G, G, G, 4))
    q = np.zeros(pl) if q is None else _arr(q, (pl,))
    u = np.zeros(pl) if u is None else _arr(u, (pl,))
    gv = np.zeros((G, G, G, 3))
    lib().orc_grid_update(ct.byref(spec), _d(g), _d(q), _d(u), _d(gv))
    return gv


def g2p(spec, st: State, gv):
    G = spec.G
    gv = _arr(gv, (G, G, G, 3))
    out = st.copy()
    status = lib().orc_g2p(ct.byref(spec), out.n, _d(out.x), _d(out.v), _d(out.C), _d(out.F), _d(gv))
    return out, status


# ------------------------------------------------------------------------ substeps / rollouts

def substep(spec, st: State, q=None, u=None, act=None):
    out = st.copy()
    pl = pose_len(spec)
    q = np.zeros(pl) if q is None else _arr(q, (pl,))
    u = np.zeros(pl) if u is None else _arr(u, (pl,))
    a = _arr(np.zeros(1) if act is None else act)
    status = lib().orc_substep(ct.byref(spec), out.n, _d(out.x), _d(out.v), _d(out.C), _d(out.F), _gp(out.group),
                               _d(q), _d(u), _d(a))
    return out, status


def substep_adj(spec, st: State, adj_end, q=None, u=None, act=None, n_act=1):
    """Adjoint of one substep.  adj_end = (xb, vb, Cb, Fb) of the end state.  Returns the
    adjoint of the start state, dL/dq, dL/du through the body velocity (pose vectors), dL/dact."""
    xb, vb, Cb, Fb = [_arr(a).copy() for a in adj_end]
    pl = pose_len(spec)
    q = np.zeros(pl) if q is None else _arr(q, (pl,))
    u = np.zeros(pl) if u is None else _arr(u, (pl,))
    a = _arr(np.zeros(max(1, n_act)) if act is None else act)
    qb, ub, ab = np.zeros(pl), np.zeros(pl), np.zeros(a.size)
    lib().orc_substep_adj(ct.byref(spec), st.n, _d(st.x), _d(st.v), _d(st.C), _d(st.F), _gp(st.group), _d(q), _d(u),
                          _d(a), _d(xb), _d(vb), _d(Cb), _d(Fb), _d(qb), _d(ub), _d(ab))
    return (xb.reshape(-1, 3), vb.reshape(-1, 3), Cb.reshape(-1, 3, 3), Fb.reshape(-1, 3, 3)), qb, ub, ab


def reward(spec, st: State, q, a):
    q, a = _arr(q, (pose_len(spec),)), _arr(a)
    return lib().orc_reward(ct.byref(spec), st.n, _d(st.x), _d(st.v), _d(q), _d(a))


def rollout(spec, st: State, q0, actions):
    """actions: (T, A).  Returns (final State, final pose, rewards (T,), status)."""
    actions = _arr(actions)
    T = actions.shape[0]
    out = st.copy()
    q = _arr(q0, (pose_len(spec),)).copy()
    rew = np.zeros(T)
    status = lib().orc_rollout(ct.byref(spec), out.n, _d(out.x), _d(out.v), _d(out.C), _d(out.F), _gp(out.group),
                               _d(q), _d(actions), T, _d(rew))
    return out, q, rew, status


def rollout_adj(spec, st: State, q0, actions, adj_final=None, rbar=None, obs_adj=None):
    """Forward + reverse.  adj_final = (xb, vb, Cb, Fb) of the final state or None;
    rbar (T,) or None; obs_adj (T + 1, obs_dim) adjoints of the observations of the states at
    the control-step boundaries, or None.  Returns (act_grad (T, A), (xb0, vb0, Cb0, Fb0), qb0)."""
    actions = _arr(actions)
    T, A = actions.shape
    n = st.n
    q0 = _arr(q0, (pose_len(spec),))
    null = ct.cast(None, _D)
    fin = [null] * 4
    keep = []
    if adj_final is not None:
        for i, a in enumerate(adj_final):
            if a is not None:
                arr = _arr(a)
                keep.append(arr)
                fin[i] = _d(arr)
    rb = null
    if rbar is not None:
        rbar = _arr(rbar)
        keep.append(rbar)
        rb = _d(rbar)
    ag = np.zeros((T, A))
    xb, vb, Cb, Fb = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3, 3)), np.zeros((n, 3, 3))
    qb = np.zeros(pose_len(spec))
    ob = null
    if obs_adj is not None:
        obs_adj = _arr(obs_adj)
        if obs_adj.shape != (T + 1, obs_dim(spec, n)):
            raise ValueError(f"obs_adj must be ({T + 1}, {obs_dim(spec, n)})")
        keep.append(obs_adj)
        ob = _d(obs_adj)
    lib().orc_rollout_adj_obs(ct.byref(spec), n, _d(st.x), _d(st.v), _d(st.C), _d(st.F), _gp(st.group), _d(q0),
                              _d(actions), T, fin[0], fin[1], fin[2], fin[3], rb, ob, _d(ag), _d(xb), _d(vb),
                              _d(Cb), _d(Fb), _d(qb))
    return ag, (xb, vb, Cb, Fb), qb


def obs_dim(spec, n):
    """Length of one environment's observation (3 n_sub + 10)."""
    return lib().orc_obs_dim(ct.byref(spec), n)


def observe(spec, x, q):
    """Observation of a state: x' of particles 0..ns-1, their mean, 4 action-driven pose
    components (zero padded), 3 target entries (reach reward, else zeros)."""
    x = _arr(x)
    n = x.shape[0]
    out = np.zeros(obs_dim(spec, n))
    lib().orc_observe(ct.byref(spec), n, _d(x), _d(_arr(q, (pose_len(spec),))), _d(out))
    return out


def bin_keys_f32(x32, G):
    x32 = np.ascontiguousarray(np.asarray(x32, np.float32).reshape(-1, 3))
    keys = np.zeros(x32.shape[0], np.uint32)
    lib().orc_bin_keys_f32(x32.shape[0], x32.ctypes.data_as(ct.POINTER(ct.c_float)), G,
                           keys.ctypes.data_as(ct.POINTER(ct.c_uint)))
    return keys


def stable_sort(keys):
    keys = np.ascontiguousarray(np.asarray(keys, np.uint32))
    perm = np.zeros(keys.size, np.uint32)
    lib().orc_stable_sort_u32(keys.size, keys.ctypes.data_as(ct.POINTER(ct.c_uint)),
                              perm.ctypes.data_as(ct.POINTER(ct.c_uint)))
    return perm
