"""ctypes binding of the FP64 tetrahedral-FEM oracle (fem_oracle.c).

TEST INFRASTRUCTURE ONLY.  Imported by tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; never by the product package.  The oracle is a plain,
single-threaded FP64 implementation of arXiv 2412.12089 App. D.2 (stable neo-Hookean
tetrahedral FEM, semi-implicit Euler) with App. E's SoftJumper damping, activations and
reward, and of its exact discrete adjoint (Sec. 4.1).

Arrays are vertex-major: x, v (n_v, 3); tets (n_t, 4) int32; group (n_t,) int32.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfem_oracle.so")
SRC = os.path.join(HERE, "fem_oracle.c")
HDR = os.path.join(HERE, "fem_oracle.h")

REWARD = {"none": 0, "jump": 3}


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < max(os.path.getmtime(SRC),
                                                                                  os.path.getmtime(HDR)):
        tmp = LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                               "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


class FemSpec(ct.Structure):
    _fields_ = [
        ("n_v", ct.c_int), ("n_t", ct.c_int), ("S", ct.c_int), ("n_act", ct.c_int), ("reward_kind", ct.c_int),
        ("n_sub", ct.c_int), ("dt", ct.c_double), ("gravity", ct.c_double * 3), ("mu", ct.c_double),
        ("lam", ct.c_double), ("alpha", ct.c_double), ("k_damp", ct.c_double), ("act_scale", ct.c_double),
        ("ground_z", ct.c_double), ("ground_mu", ct.c_double), ("rparam", ct.c_double * 4),
    ]


_lib = None
_D = ct.POINTER(ct.c_double)
_I = ct.POINTER(ct.c_int)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ct.CDLL(LIB_PATH)
        P = ct.POINTER(FemSpec)
        L.fem_rest.argtypes = [P, _I, _D, ct.c_double, _D, _D, _D]
        L.fem_rest.restype = ct.c_int
        L.fem_psi.argtypes = [P, _D, ct.c_double]
        L.fem_psi.restype = ct.c_double
        L.fem_stress.argtypes = [P, _D, ct.c_double, _D]
        L.fem_stress_vjp.argtypes = [P, _D, ct.c_double, _D, _D, _D]
        L.fem_energy.argtypes = [P, _I, _D, _D, _D, _D]
        L.fem_energy.restype = ct.c_double
        L.fem_forces.argtypes = [P, _I, _D, _D, _D, _D, _D, _D]
        L.fem_substep.argtypes = [P, _I, _D, _D, _D, _D, _D, _D]
        L.fem_substep.restype = ct.c_int
        L.fem_rollout.argtypes = [P, _I, _I, _D, _D, _D, _D, _D, _D, ct.c_int, _D]
        L.fem_rollout.restype = ct.c_int
        L.fem_rollout_adj.argtypes = [P, _I, _I, _D, _D, _D, _D, _D, _D, ct.c_int, _D, _D, _D, _D, _D, _D]
        L.fem_rollout_adj.restype = ct.c_int
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _i(a):
    return a.ctypes.data_as(_I)


def _f64(a, shape=None):
    out = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return out.reshape(shape) if shape is not None else out


def _opt(a, shape):
    return None if a is None else _f64(a, shape)


def lame(E, nu):
    return E / (2.0 * (1.0 + nu)), E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))


class Mesh:
    """A spec plus its mesh and rest quantities (Dm^-1, rest volumes, inverse masses)."""

    def __init__(self, spec: FemSpec, tets, group, rest_x, rho):
        self.spec = spec
        self.tets = np.ascontiguousarray(np.asarray(tets, np.int32).reshape(-1, 4))
        self.group = np.ascontiguousarray(np.asarray(group, np.int32).reshape(-1))
        self.rest_x = _f64(rest_x, (-1, 3))
        n_t, n_v = self.tets.shape[0], self.rest_x.shape[0]
        assert spec.n_t == n_t and spec.n_v == n_v
        self.dminv = np.zeros((n_t, 9))
        self.vol = np.zeros(n_t)
        self.inv_mass = np.zeros(n_v)
        rc = lib().fem_rest(ct.byref(spec), _i(self.tets), _d(self.rest_x), float(rho), _d(self.dminv),
                            _d(self.vol), _d(self.inv_mass))
        if rc != 0:
            raise ValueError("degenerate element")

    def _args(self):
        return ct.byref(self.spec), _i(self.tets)


def make_mesh(es) -> Mesh:
    """Mesh from a workloads.EnvSpec with material "fem"."""
    mu, lam = lame(es.E, es.nu)
    s = FemSpec()
    s.n_v, s.n_t = es.n_particles, int(np.asarray(es.fem_tets).reshape(-1, 4).shape[0])
    s.S, s.n_act = es.substeps, es.n_groups
    s.reward_kind = REWARD[es.reward]
    s.n_sub = es.n_sub
    s.dt = es.dt
    for k in range(3):
        s.gravity[k] = es.gravity[k]
    s.mu, s.lam, s.alpha = mu, lam, 0.0
    s.k_damp, s.act_scale = es.k_damp, es.act_stress
    s.ground_z, s.ground_mu = es.ground_z, es.ground_mu
    for k in range(4):
        s.rparam[k] = es.rparam[k]
    return Mesh(s, es.fem_tets, es.fem_group, es.fem_rest, es.rho)


def spec(n_v, n_t, **kw) -> FemSpec:
    s = FemSpec()
    s.n_v, s.n_t = n_v, n_t
    s.S, s.n_act, s.reward_kind, s.n_sub = kw.get("S", 1), kw.get("n_act", 0), kw.get("reward_kind", 0), kw.get(
        "n_sub", n_v)
    s.dt = kw.get("dt", 1e-3)
    g = kw.get("gravity", (0.0, 0.0, -9.8))
    for k in range(3):
        s.gravity[k] = g[k]
    s.mu, s.lam, s.alpha = kw.get("mu", 1000.0), kw.get("lam", 1000.0), kw.get("alpha", 0.0)
    s.k_damp, s.act_scale = kw.get("k_damp", 0.0), kw.get("act_scale", 0.0)
    s.ground_z, s.ground_mu = kw.get("ground_z", -1e9), kw.get("ground_mu", 0.0)
    rp = kw.get("rparam", (0.0, 0.0, 0.0, 0.0))
    for k in range(4):
        s.rparam[k] = rp[k]
    return s


def psi(s, F, a=0.0):
    return lib().fem_psi(ct.byref(s), _d(_f64(F, 9)), float(a))


def stress(s, F, a=0.0):
    P = np.zeros(9)
    lib().fem_stress(ct.byref(s), _d(_f64(F, 9)), float(a), _d(P))
    return P.reshape(3, 3)


def stress_vjp(s, F, a, Pb):
    Fb = np.zeros(9)
    ab = np.zeros(1)
    lib().fem_stress_vjp(ct.byref(s), _d(_f64(F, 9)), float(a), _d(_f64(Pb, 9)), _d(Fb), _d(ab))
    return Fb.reshape(3, 3), float(ab[0])


def energy(m: Mesh, x, a_elem=None):
    ae = _opt(a_elem, -1)
    return lib().fem_energy(ct.byref(m.spec), _i(m.tets), _d(m.dminv), _d(m.vol), _d(_f64(x, (-1, 3))),
                            _d(ae) if ae is not None else None)


def forces(m: Mesh, x, v, a_elem=None):
    f = np.zeros((m.spec.n_v, 3))
    ae = _opt(a_elem, -1)
    lib().fem_forces(ct.byref(m.spec), _i(m.tets), _d(m.dminv), _d(m.vol), _d(_f64(x, (-1, 3))),
                     _d(_f64(v, (-1, 3))), _d(ae) if ae is not None else None, _d(f))
    return f


def substep(m: Mesh, x, v, a_elem=None):
    x, v = _f64(x, (-1, 3)).copy(), _f64(v, (-1, 3)).copy()
    ae = _opt(a_elem, -1)
    st = lib().fem_substep(ct.byref(m.spec), _i(m.tets), _d(m.dminv), _d(m.vol), _d(m.inv_mass), _d(x), _d(v),
                           _d(ae) if ae is not None else None)
    return x, v, st


def rollout(m: Mesh, x0, v0, actions):
    x, v = _f64(x0, (-1, 3)).copy(), _f64(v0, (-1, 3)).copy()
    T = int(np.asarray(actions).shape[0]) if m.spec.n_act > 0 else int(np.asarray(actions).shape[0])
    acts = _f64(actions, (T, max(m.spec.n_act, 1)))
    if m.spec.n_act == 0:
        acts = np.zeros((T, 1))
    r = np.zeros(T)
    st = lib().fem_rollout(ct.byref(m.spec), _i(m.tets), _i(m.group), _d(m.dminv), _d(m.vol), _d(m.inv_mass), _d(x),
                           _d(v), _d(acts), T, _d(r))
    return x, v, r, st


def rollout_adj(m: Mesh, x0, v0, actions, xbT=None, vbT=None, rbar=None):
    T = int(np.asarray(actions).shape[0])
    A = max(m.spec.n_act, 1)
    acts = _f64(actions, (T, A)) if m.spec.n_act > 0 else np.zeros((T, 1))
    ag = np.zeros((T, A))
    xb0 = np.zeros((m.spec.n_v, 3))
    vb0 = np.zeros((m.spec.n_v, 3))
    xb = _opt(xbT, (-1, 3))
    vb = _opt(vbT, (-1, 3))
    rb = _opt(rbar, -1)
    st = lib().fem_rollout_adj(ct.byref(m.spec), _i(m.tets), _i(m.group), _d(m.dminv), _d(m.vol), _d(m.inv_mass),
                               _d(_f64(x0, (-1, 3))), _d(_f64(v0, (-1, 3))), _d(acts), T,
                               _d(xb) if xb is not None else None, _d(vb) if vb is not None else None,
                               _d(rb) if rb is not None else None, _d(ag), _d(xb0), _d(vb0))
    return ag[:, :m.spec.n_act], xb0, vb0, st
