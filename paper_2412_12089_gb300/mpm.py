"""ctypes binding of the C ABI in include/mpm.h (argument marshalling only).

Every function here has the name of the C entry point it calls and only converts
arguments: torch tensors / numpy arrays to pointers, EnvSpec dataclasses to the C
struct, status codes to exceptions.  All simulation work runs in the CUDA library
``libmpm_gb300.so``; if it is missing or cannot be loaded, importing the functions
raises - there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmpm_gb300.so")

MAT = {"neohookean": 0, "vonmises": 1, "fluid": 2, "muscle": 3, "fem": 4}
COLL = {"none": 0, "capsule": 1, "box": 2, "container": 3, "capsules": 4}
REWARD = {"none": 0, "flat": 1, "reach": 2, "jump": 3}
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "NUMERIC", 5: "DOMAIN", 6: "TIMEOUT",
          7: "NOT_READY", 8: "BUDGET", 9: "STATE"}
MPM_OK, MPM_NOT_READY = 0, 7
MPM_STEP_RECORD = 1
# per-environment status word masks (mpm_check_status)
MPM_FLAG_DOMAIN, MPM_FLAG_NAN, MPM_FLAG_INVERTED, MPM_FLAG_WAIT = 0x1, 0x2, 0x4, 0x8


class MpmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mpm status {STATUS.get(code, code)}: {msg}")
        self.code = code


class MpmEnvSpec(ct.Structure):
    _fields_ = [
        ("n_particles", ct.c_int32), ("grid_res", ct.c_int32), ("substeps", ct.c_int32), ("bound", ct.c_int32),
        ("material", ct.c_int32), ("collider", ct.c_int32), ("n_coll_act", ct.c_int32),
        ("act_map", ct.c_int32 * 4), ("n_groups", ct.c_int32), ("reward", ct.c_int32), ("n_sub", ct.c_int32),
        ("dt", ct.c_float), ("gravity", ct.c_float * 3), ("E", ct.c_float), ("nu", ct.c_float),
        ("rho", ct.c_float), ("p_vol", ct.c_float), ("yield_stress", ct.c_float), ("c_y", ct.c_float),
        ("bulk", ct.c_float), ("visc", ct.c_float), ("act_stress", ct.c_float), ("coll_dims", ct.c_float * 4),
        ("coll_mu", ct.c_float), ("alpha", ct.c_float), ("act_scale", ct.c_float * 4), ("ground_mu", ct.c_float),
        ("rparam", ct.c_float * 4), ("pose0", ct.c_float * 4), ("n_caps", ct.c_int32),
        ("cap_offset", ct.c_float * 3), ("n_tets", ct.c_int32), ("fem_tets", ct.c_void_p),
        ("fem_rest", ct.c_void_p), ("fem_group", ct.c_void_p), ("k_damp", ct.c_float), ("ground_z", ct.c_float),
    ]


class MpmOptions(ct.Structure):
    _fields_ = [("max_steps", ct.c_int32), ("per_env_launch", ct.c_int32), ("use_graphs", ct.c_int32),
                ("chunk", ct.c_int32), ("device", ct.c_int32), ("grid_tape_fraction", ct.c_float),
                ("keep_fraction", ct.c_float)]


class MpmServerOptions(ct.Structure):
    _fields_ = [("mem_fraction", ct.c_double), ("max_resident", ct.c_int32), ("device", ct.c_int32),
                ("chunk", ct.c_int32)]


class MpmRequest(ct.Structure):
    _fields_ = [("spec", MpmEnvSpec), ("x", ct.c_void_p), ("v", ct.c_void_p), ("C", ct.c_void_p),
                ("F", ct.c_void_p), ("group", ct.c_void_p), ("horizon", ct.c_int32), ("actions", ct.c_void_p),
                ("want_grad", ct.c_int32), ("reward_adj", ct.c_void_p)]


class MpmResult(ct.Structure):
    _fields_ = [("status", ct.c_int32), ("horizon", ct.c_int32), ("action_dim", ct.c_int32),
                ("n_particles", ct.c_int32), ("rewards", ct.POINTER(ct.c_float)),
                ("action_grad", ct.POINTER(ct.c_float)), ("x_final", ct.POINTER(ct.c_float)),
                ("submit_ms", ct.c_double), ("admit_ms", ct.c_double), ("finish_ms", ct.c_double)]


_lib = None
_P = ct.c_void_p


def lib():
    """Load libmpm_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is missing; build it with __graft_entry__.build()")
    L = ct.CDLL(LIB_PATH)
    i32, i64, u32 = ct.c_int32, ct.c_int64, ct.c_uint32
    sig = {
        "mpm_create": (i32, [ct.POINTER(MpmEnvSpec), ct.c_int, ct.POINTER(MpmOptions), ct.POINTER(_P)]),
        "mpm_destroy": (None, [_P]),
        "mpm_n_envs": (i32, [_P]),
        "mpm_n_particles": (i64, [_P]),
        "mpm_action_dim": (i32, [_P]),
        "mpm_tape_length": (i32, [_P]),
        "mpm_device_bytes": (i64, [_P]),
        "mpm_kept_steps": (i32, [_P]),
        "mpm_last_error": (ct.c_char_p, [_P]),
        "mpm_set_state": (i32, [_P, _P, _P, _P, _P, _P, _P, _P]),
        "mpm_get_state": (i32, [_P, _P, _P, _P, _P, _P, _P]),
        "mpm_step": (i32, [_P, _P, _P, u32, _P]),
        "mpm_backward": (i32, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
        "mpm_backward_begin": (i32, [_P, _P, _P, _P, _P, _P]),
        "mpm_backward_step": (i32, [_P, _P, _P, _P, ct.POINTER(ct.c_int32), _P]),
        "mpm_backward_end": (i32, [_P, _P, _P, _P, _P, _P, _P, _P]),
        "mpm_reset_tape": (i32, [_P]),
        "mpm_check_status": (i32, [_P, _P]),
        "mpm_bin": (i32, [_P, i32, i32, _P, _P, _P]),
        "mpm_bin_static": (i32, [_P, i32, i32, _P, _P, _P]),
        "mpm_autotune": (i32, [_P, i32, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_float)]),
        "mpm_autotune_config": (i32, [_P, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_float), ct.POINTER(ct.c_int32),
                                      ct.POINTER(ct.c_float)]),
        "mpm_obs_dim": (i32, [_P]),
        "mpm_observe": (i32, [_P, _P, _P]),
        "mpm_set_obs_adjoint": (i32, [_P, _P, _P]),
        "mpm_bin_static_max": (i32, []),
        "mpm_kernel_launches": (i64, [_P]),
        "mpm_time_kernel": (i32, [_P, i32]),
        "mpm_kernel_time": (i32, [_P, ct.POINTER(ct.c_double), ct.POINTER(ct.c_int64)]),
        "mpm_last_active_tiles": (i32, [_P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    if hasattr(L, "mpm_server_create"):
        ssig = {
            "mpm_server_create": (i32, [ct.POINTER(MpmServerOptions), ct.POINTER(_P)]),
            "mpm_server_destroy": (None, [_P]),
            "mpm_submit": (i32, [_P, ct.POINTER(MpmRequest), ct.POINTER(ct.c_uint64)]),
            "mpm_poll": (i32, [_P, ct.c_uint64, ct.POINTER(MpmResult)]),
            "mpm_wait": (i32, [_P, ct.c_uint64, ct.c_double, ct.POINTER(MpmResult)]),
            "mpm_release": (i32, [_P, ct.c_uint64]),
            "mpm_server_last_error": (ct.c_char_p, [_P]),
        }
        for name, (res, args) in ssig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
    _lib = L
    return L


# ----------------------------------------------------------------------------- marshalling

def ptr(a):
    """Pointer of a torch tensor / numpy array (contiguous), or None."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def stream_ptr(stream):
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


def to_c_spec(es) -> MpmEnvSpec:
    """MpmEnvSpec from a workloads.EnvSpec."""
    s = MpmEnvSpec()
    s.n_particles, s.grid_res, s.substeps, s.bound = es.n_particles, es.grid_res, es.substeps, es.bound
    s.material, s.collider, s.reward = MAT[es.material], COLL[es.collider], REWARD[es.reward]
    s.n_coll_act = es.n_coll_act
    s.n_caps = es.n_caps if es.collider == "capsules" else 0
    for i in range(3):
        s.cap_offset[i] = es.cap_offset[i]
    for j in range(4):
        s.act_map[j] = es.act_map[j] if j < len(es.act_map) else 0
        s.act_scale[j] = es.act_scale[j] if j < len(es.act_scale) else 0.0
        s.coll_dims[j] = es.coll_dims[j]
        s.rparam[j] = es.rparam[j]
        s.pose0[j] = es.pose0[j]
    s.n_groups, s.n_sub = es.n_groups, es.n_sub
    s.dt = es.dt
    for i in range(3):
        s.gravity[i] = es.gravity[i]
    s.E, s.nu, s.rho, s.p_vol = es.E, es.nu, es.rho, es.p_vol
    s.yield_stress, s.c_y = es.yield_stress, es.c_y
    s.bulk, s.visc, s.act_stress = es.bulk, es.visc, es.act_stress
    s.coll_mu, s.alpha, s.ground_mu = es.coll_mu, es.alpha, es.ground_mu
    s.k_damp, s.ground_z = getattr(es, "k_damp", 0.0), getattr(es, "ground_z", 0.0)
    if es.material == "fem":
        # the struct points into these arrays: keep them alive as long as the struct
        tets = np.ascontiguousarray(np.asarray(es.fem_tets, np.int32).reshape(-1, 4))
        rest = np.ascontiguousarray(np.asarray(es.fem_rest, np.float32).reshape(-1, 3))
        grp = None if es.fem_group is None else np.ascontiguousarray(np.asarray(es.fem_group, np.int32))
        s.n_tets = tets.shape[0]
        s.fem_tets, s.fem_rest = tets.ctypes.data, rest.ctypes.data
        s.fem_group = grp.ctypes.data if grp is not None else None
        s._keep = (tets, rest, grp)
    return s


def check(code, ctx=None, srv=None):
    if code != MPM_OK:
        msg = ""
        if ctx is not None:
            msg = (lib().mpm_last_error(ctx) or b"").decode()
        elif srv is not None:
            msg = (lib().mpm_server_last_error(srv) or b"").decode()
        raise MpmError(code, msg)
    return code


# ----------------------------------------------------------------------------- same-name wrappers

def mpm_create(specs, max_steps=0, per_env_launch=False, use_graphs=True, chunk=0, device=0, grid_tape_fraction=0.0,
               keep_fraction=0.0):
    cs = [to_c_spec(s) if not isinstance(s, MpmEnvSpec) else s for s in specs]  # alive through the call
    arr = (MpmEnvSpec * len(specs))(*cs)
    opt = MpmOptions(max_steps, 1 if per_env_launch else 0, 1 if use_graphs else 0, chunk, device, grid_tape_fraction,
                     keep_fraction)
    h = _P()
    code = lib().mpm_create(arr, len(specs), ct.byref(opt), ct.byref(h))
    if code != MPM_OK:
        msg = (lib().mpm_last_error(h) or b"").decode() if h.value else ""
        if h.value:
            lib().mpm_destroy(h)
        raise MpmError(code, msg)
    return h


def mpm_destroy(ctx):
    lib().mpm_destroy(ctx)


def mpm_set_state(ctx, x, v, C, F, group=None, pose=None, stream=None):
    return check(lib().mpm_set_state(ctx, ptr(x), ptr(v), ptr(C), ptr(F), ptr(group), ptr(pose), stream_ptr(stream)),
                 ctx)


def mpm_get_state(ctx, x=None, v=None, C=None, F=None, pose=None, stream=None):
    return check(lib().mpm_get_state(ctx, ptr(x), ptr(v), ptr(C), ptr(F), ptr(pose), stream_ptr(stream)), ctx)


def mpm_step(ctx, actions, reward=None, flags=0, stream=None):
    return check(lib().mpm_step(ctx, ptr(actions), ptr(reward), flags, stream_ptr(stream)), ctx)


def mpm_backward(ctx, xb=None, vb=None, Cb=None, Fb=None, reward_adj=None, action_grad=None, xb0=None, vb0=None,
                 Cb0=None, Fb0=None, pose_grad0=None, stream=None):
    return check(lib().mpm_backward(ctx, ptr(xb), ptr(vb), ptr(Cb), ptr(Fb), ptr(reward_adj), ptr(action_grad),
                                    ptr(xb0), ptr(vb0), ptr(Cb0), ptr(Fb0), ptr(pose_grad0), stream_ptr(stream)), ctx)


def mpm_backward_begin(ctx, xb=None, vb=None, Cb=None, Fb=None, stream=None):
    return check(lib().mpm_backward_begin(ctx, ptr(xb), ptr(vb), ptr(Cb), ptr(Fb), stream_ptr(stream)), ctx)


def mpm_backward_step(ctx, reward_adj=None, obs_adj=None, action_grad=None, stream=None):
    """Reverse the next recorded step; returns its index t."""
    t = ct.c_int32(-1)
    check(lib().mpm_backward_step(ctx, ptr(reward_adj), ptr(obs_adj), ptr(action_grad), ct.byref(t),
                                  stream_ptr(stream)), ctx)
    return t.value


def mpm_backward_end(ctx, obs_adj=None, xb0=None, vb0=None, Cb0=None, Fb0=None, pose_grad0=None, stream=None):
    return check(lib().mpm_backward_end(ctx, ptr(obs_adj), ptr(xb0), ptr(vb0), ptr(Cb0), ptr(Fb0), ptr(pose_grad0),
                                        stream_ptr(stream)), ctx)


def mpm_reset_tape(ctx):
    return check(lib().mpm_reset_tape(ctx), ctx)


def mpm_check_status(ctx, n_envs):
    flags = np.zeros(n_envs, np.int32)
    code = lib().mpm_check_status(ctx, flags.ctypes.data)
    return code, flags


def mpm_bin(x, n, grid_res, keys, perm, stream=None):
    code = lib().mpm_bin(ptr(x), n, grid_res, ptr(keys), ptr(perm), stream_ptr(stream))
    if code != MPM_OK:
        raise MpmError(code, "mpm_bin")
    return code


def mpm_bin_static(x, n, grid_res, keys, perm, stream=None):
    code = lib().mpm_bin_static(ptr(x), n, grid_res, ptr(keys), ptr(perm), stream_ptr(stream))
    if code != MPM_OK:
        raise MpmError(code, "mpm_bin_static")
    return code


def mpm_bin_static_max():
    return lib().mpm_bin_static_max()


def mpm_autotune(ctx, trials=3):
    """Pick the scatter shape per material on the current state; returns
    ({material: capacity}, {material: (ms with 512, 1024, 256)}) for materials present."""
    box = (ct.c_int32 * 4)()
    ms = (ct.c_float * 12)()
    check(lib().mpm_autotune(ctx, trials, box, ms), ctx=ctx)
    names = ("neohookean", "vonmises", "fluid", "muscle")
    chosen = {names[m]: int(box[m]) for m in range(4) if box[m]}
    times = {names[m]: tuple(float(ms[3 * m + b]) for b in range(3)) for m in range(4) if box[m]}
    return chosen, times


def mpm_autotune_config(ctx):
    """The rest of the autotuner's choice: {"grid_blocks", "grid_ms" (per CTA choice),
    "g2p_stage" {material: 0/1}, "g2p_ms" {material: (ms without, ms with staging)}}."""
    gb = ct.c_int32()
    gms = (ct.c_float * 4)()
    st = (ct.c_int32 * 4)()
    sms = (ct.c_float * 8)()
    check(lib().mpm_autotune_config(ctx, ct.byref(gb), gms, st, sms), ctx=ctx)
    names = ("neohookean", "vonmises", "fluid", "muscle")
    return {"grid_blocks": int(gb.value), "grid_ms_304_608_1216_2432": [float(v) for v in gms],
            "g2p_stage": {names[m]: int(st[m]) for m in range(4) if st[m] >= 0},
            "g2p_ms_plain_staged": {names[m]: (float(sms[2 * m]), float(sms[2 * m + 1])) for m in range(4) if st[m] >= 0}}


def mpm_obs_dim(ctx):
    return lib().mpm_obs_dim(ctx)


def mpm_observe(ctx, obs, stream=None):
    return check(lib().mpm_observe(ctx, ptr(obs), stream_ptr(stream)), ctx=ctx)


def mpm_set_obs_adjoint(ctx, obs_adj, stream=None):
    return check(lib().mpm_set_obs_adjoint(ctx, ptr(obs_adj), stream_ptr(stream)), ctx=ctx)


def mpm_tape_length(ctx):
    return lib().mpm_tape_length(ctx)


def mpm_device_bytes(ctx):
    return lib().mpm_device_bytes(ctx)


def mpm_kept_steps(ctx):
    return lib().mpm_kept_steps(ctx)


KERNEL_CLASS = {"p2g": 1, "grid": 2, "g2p": 3, "g2p_adj": 4, "grid_adj": 5, "p2g_adj": 6, "bin": 7, "other": 8}


def mpm_kernel_launches(ctx):
    return lib().mpm_kernel_launches(ctx)


def mpm_time_kernel(ctx, kernel_class):
    if kernel_class == "all":
        kernel_class = -1
    kc = KERNEL_CLASS[kernel_class] if isinstance(kernel_class, str) else int(kernel_class)
    return check(lib().mpm_time_kernel(ctx, kc), ctx)


def mpm_kernel_time(ctx, all_classes=False):
    """(total_ms, launches) of the timed class, or dicts by class name when all were timed."""
    k = len(KERNEL_CLASS) + 1
    ms = (ct.c_double * k)()
    n = (ct.c_int64 * k)()
    check(lib().mpm_kernel_time(ctx, ms, n), ctx)
    if not all_classes:
        return ms[0], n[0]
    return ({name: ms[i] for name, i in KERNEL_CLASS.items()}, {name: n[i] for name, i in KERNEL_CLASS.items()})


def mpm_last_active_tiles(ctx):
    return lib().mpm_last_active_tiles(ctx)


# ----------------------------------------------------------------------------- serving

def mpm_server_create(mem_fraction=0.8, max_resident=64, device=0, chunk=0):
    opt = MpmServerOptions(mem_fraction, max_resident, device, chunk)
    h = _P()
    code = lib().mpm_server_create(ct.byref(opt), ct.byref(h))
    if code != MPM_OK:
        raise MpmError(code, "mpm_server_create")
    return h


def mpm_server_destroy(srv):
    lib().mpm_server_destroy(srv)


def mpm_submit(srv, spec, init, actions, horizon, want_grad=False, reward_adj=None):
    """Submit one rollout request (host arrays are copied before this returns)."""
    x = np.ascontiguousarray(init.x, np.float32)
    v = np.ascontiguousarray(init.v, np.float32)
    C = np.ascontiguousarray(init.C, np.float32)
    F = np.ascontiguousarray(init.F, np.float32)
    g = np.ascontiguousarray(init.group, np.int32) if init.group is not None else None
    a = np.ascontiguousarray(actions, np.float32).reshape(horizon, -1) if actions is not None else None
    rb = np.ascontiguousarray(reward_adj, np.float32) if reward_adj is not None else None
    req = MpmRequest()
    cspec = to_c_spec(spec)  # alive through the call (FEM mesh arrays)
    req.spec = cspec
    req.x, req.v, req.C, req.F = x.ctypes.data, v.ctypes.data, C.ctypes.data, F.ctypes.data
    req.group = g.ctypes.data if g is not None else None
    req.horizon = horizon
    req.actions = a.ctypes.data if a is not None else None
    req.want_grad = 1 if want_grad else 0
    req.reward_adj = rb.ctypes.data if rb is not None else None
    t = ct.c_uint64()
    check(lib().mpm_submit(srv, ct.byref(req), ct.byref(t)), srv=srv)
    return t.value


def _result(res):
    out = {"status": res.status, "horizon": res.horizon, "submit_ms": res.submit_ms, "admit_ms": res.admit_ms,
           "finish_ms": res.finish_ms}
    T, A, n = res.horizon, res.action_dim, res.n_particles
    out["rewards"] = np.ctypeslib.as_array(res.rewards, (T,)).copy() if res.rewards else None
    out["action_grad"] = np.ctypeslib.as_array(res.action_grad, (T, A)).copy() if (res.action_grad and A) else None
    out["x_final"] = np.ctypeslib.as_array(res.x_final, (n, 3)).copy() if res.x_final else None
    return out


def mpm_poll(srv, ticket):
    """None while the request runs, else its result dict."""
    res = MpmResult()
    code = lib().mpm_poll(srv, ticket, ct.byref(res))
    if code == MPM_NOT_READY:
        return None
    check(code, srv=srv)
    return _result(res)


def mpm_wait(srv, ticket, timeout_ms=60000.0):
    res = MpmResult()
    check(lib().mpm_wait(srv, ticket, timeout_ms, ct.byref(res)), srv=srv)
    return _result(res)


def mpm_release(srv, ticket):
    return check(lib().mpm_release(srv, ticket), srv=srv)
