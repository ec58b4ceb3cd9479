"""Seeded synthetic inputs for the batched MPM path.

This module only draws random numbers and lays out initial states; it holds none of
the method's arithmetic.  Both the CUDA path (through the C ABI) and the FP64 oracle
(in tests and the CPU-baseline leg of the benchmark) take their inputs from here, so
both see the same FP32-representable values.

The shapes follow the paper's deformable tasks (arXiv 2412.12089, App. E): RollingFlat
(elastoplastic dough under a rolling pin, 48^3 grid), FluidMove (fluid in a moving
container), SoftJumper (as an MPM solid with active fibres, and as the paper's tetrahedral
FEM quadruped), HandFlip (a slab on driven capsule fingers), and a neo-Hookean cube for the
single-environment case.  The task assets (PlasticineLab dough meshes,
SoftGym containers, the Shadow hand) are not available, so each is replaced by a
parametric stand-in with the paper's sizes, materials and time steps.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np

MATERIALS = ("neohookean", "vonmises", "fluid", "muscle", "fem")
COLLIDERS = ("none", "capsule", "box", "container", "capsules")
REWARDS = ("none", "flat", "reach", "jump")


@dataclass
class EnvSpec:
    """Physical description of one environment (inputs only)."""

    n_particles: int
    grid_res: int
    substeps: int
    dt: float
    material: str = "neohookean"
    E: float = 1e4
    nu: float = 0.3
    rho: float = 1e3
    p_vol: float = 1e-6
    yield_stress: float = 0.0
    c_y: float = 2.0
    bulk: float = 0.0
    visc: float = 0.0
    act_stress: float = 0.0
    gravity: tuple = (0.0, 0.0, -9.8)
    bound: int = 3
    collider: str = "none"
    coll_dims: tuple = (0.0, 0.0, 0.0, 0.0)
    coll_mu: float = 0.0
    alpha: float = 666.0
    act_map: tuple = ()
    act_scale: tuple = ()
    n_groups: int = 0
    ground_mu: float = 0.0
    reward: str = "none"
    n_sub: int = 250
    rparam: tuple = (0.0, 0.0, 0.0, 0.0)
    pose0: tuple = (0.0, 0.0, 0.0, 0.0)
    n_caps: int = 0                       # collider "capsules": capsules of coll_dims (1..8)
    cap_offset: tuple = (0.0, 0.0, 0.0)   # initial position of capsule j: pose0 + j * cap_offset
    # material "fem": a tetrahedral mesh whose vertices are the environment's particles
    k_damp: float = 0.0                   # viscous damping stress k_damp dF/dt
    ground_z: float = 0.0                 # height of the ground plane
    fem_tets: np.ndarray = None           # (n_t, 4) int32 vertex indices
    fem_rest: np.ndarray = None           # (n_particles, 3) float32 rest positions
    fem_group: np.ndarray = None          # (n_t,) int32 action index of each element

    def __post_init__(self):
        # Every real-valued input is made FP32-representable, so the FP32 CUDA path and the
        # FP64 oracle start from identical parameters.
        for f in dataclasses.fields(self):
            v = getattr(self, f.name)
            if isinstance(v, float):
                object.__setattr__(self, f.name, float(np.float32(v)))
            elif isinstance(v, tuple) and v and all(isinstance(a, float) for a in v):
                object.__setattr__(self, f.name, tuple(float(np.float32(a)) for a in v))

    @property
    def n_coll_act(self) -> int:
        """Actions that move the collider (4 per capsule for the multi-capsule collider)."""
        return 4 * self.n_caps if self.collider == "capsules" else len(self.act_map)

    @property
    def action_dim(self) -> int:
        return self.n_coll_act + self.n_groups

    def replace(self, **kw) -> "EnvSpec":
        return dataclasses.replace(self, **kw)


@dataclass
class EnvInit:
    """Initial particle state of one environment, FP32-representable values."""

    x: np.ndarray  # (n, 3) float32
    v: np.ndarray  # (n, 3) float32
    C: np.ndarray  # (n, 3, 3) float32
    F: np.ndarray  # (n, 3, 3) float32
    group: np.ndarray = field(default=None)  # (n,) int32, -1 = passive

    def __post_init__(self):
        if self.group is None:
            self.group = np.full(self.x.shape[0], -1, np.int32)


@dataclass
class Workload:
    name: str
    specs: list
    inits: list
    actions: np.ndarray  # (T, n_envs, A_max) float32
    T: int

    @property
    def n_envs(self) -> int:
        return len(self.specs)

    @property
    def n_particles(self) -> int:
        return int(sum(s.n_particles for s in self.specs))


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _rest_state(x, v, rng=None):
    n = x.shape[0]
    C = np.zeros((n, 3, 3), np.float32)
    F = np.broadcast_to(np.eye(3, dtype=np.float32), (n, 3, 3)).copy()
    return EnvInit(_f32(x), _f32(v), C, F)


def _box_points(rng, n, lo, hi):
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    return lo + (hi - lo) * rng.random((n, 3))


def _pad_actions(per_env, T):
    amax = max(1, max(a.shape[1] for a in per_env))
    out = np.zeros((T, len(per_env), amax), np.float32)
    for e, a in enumerate(per_env):
        out[:, e, : a.shape[1]] = a
    return out


# ----------------------------------------------------------------------------- C1

def cube(seed: int = 0, n: int = 4096, G: int = 32, substeps: int = 50, T: int = 1,
         vstd: float = 0.1) -> Workload:
    """Neo-Hookean cube: n particles uniform in [0.4, 0.6]^3, v ~ N(0, vstd), E=1e4,
    nu=0.3, rho=1e3, dt=1e-4, gravity, no collider."""
    rng = np.random.default_rng(seed)
    x = _box_points(rng, n, (0.4, 0.4, 0.4), (0.6, 0.6, 0.6))
    v = rng.normal(0.0, vstd, (n, 3))
    spec = EnvSpec(n_particles=n, grid_res=G, substeps=substeps, dt=1e-4, material="neohookean",
                   E=1e4, nu=0.3, rho=1e3, p_vol=0.2 ** 3 / n)
    init = _rest_state(x, v)
    return Workload("cube", [spec], [init], np.zeros((T, 1, 1), np.float32), T)


# ----------------------------------------------------------------------------- C2

def dough(n_envs: int = 512, seed: int = 0, n_range=(2000, 16000), G: int = 48, substeps: int = 20,
          T: int = 32, action_std: float = 0.5) -> Workload:
    """Von Mises elastoplastic dough (E=5e3, nu=0.2, sigma_y=50, rho=1) under a capsule
    rolling pin driven by 3-DoF relative-pose actions (p_x, p_z, theta_z) ~ N(0, 0.5).
    Particle counts are log-uniform in n_range; block 0.2 x 0.2 x 0.1 with the paper's
    x0.9-1.1 scale and +-0.1 (x, y), 0-0.05 (z) offsets."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / G
    specs, inits, acts = [], [], []
    for e in range(n_envs):
        n = int(round(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1])))))
        sc = rng.uniform(0.9, 1.1)
        size = np.array([0.2, 0.2, 0.1]) * sc
        off = np.array([rng.uniform(-0.1, 0.1), rng.uniform(-0.1, 0.1), rng.uniform(0.0, 0.05)])
        z0 = 3 * dx + 0.5 * dx
        lo = np.array([0.5 - size[0] / 2, 0.5 - size[1] / 2, z0]) + off
        hi = lo + size
        x = _box_points(rng, n, lo, hi)
        v = np.zeros((n, 3))
        top = hi[2]
        pose0 = (0.5 + off[0], 0.5 + off[1], top + 0.03 + 0.5 * dx, 0.0)
        spec = EnvSpec(n_particles=n, grid_res=G, substeps=substeps, dt=5e-5, material="vonmises",
                       E=5e3, nu=0.2, rho=1.0, p_vol=float(np.prod(size)) / n, yield_stress=50.0,
                       c_y=2.0, collider="capsule", coll_dims=(0.03, 0.12, 0.0, 0.0), coll_mu=0.9,
                       alpha=666.0, act_map=(0, 2, 3), act_scale=(0.005, 0.005, 0.05),
                       ground_mu=0.9, reward="flat", n_sub=min(250, n), rparam=(0.125, 0, 0, 0),
                       pose0=tuple(float(p) for p in pose0))
        specs.append(spec)
        inits.append(_rest_state(x, v))
        acts.append(rng.normal(0.0, action_std, (T, 3)))
    return Workload("dough", specs, inits, _pad_actions(acts, T), T)


# ----------------------------------------------------------------------------- C3

def fluid(n_envs: int = 1024, seed: int = 0, n: int = 8192, G: int = 64, substeps: int = 25,
          T: int = 16, action_std: float = 0.5, dt: float = 5e-4, floor_cells: float = 2.37,
          az: float = 0.1) -> Workload:
    """Weakly compressible fluid (bulk 1e4, viscosity 1e-3, rho=1e3), n particles filling
    the lower half of an open-top container (inner 0.2^3, wall 2 dx) that follows
    3-DoF translation actions ~ N(0, 0.5); reward = FluidMove's R_d to a seeded target.
    The container floor's top face starts floor_cells cells above the wall layer (3 dx) plus
    the wall thickness: the default keeps it off the node lattice; an integer, with an inner
    half-height az that is a whole number of cells, puts it on it exactly in FP32."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / G
    a, w = 0.1, 2 * dx
    specs, inits, acts = [], [], []
    for e in range(n_envs):
        # cavity centre
        c = np.array([0.5 + rng.uniform(-0.05, 0.05), 0.5 + rng.uniform(-0.05, 0.05),
                      3 * dx + w + az + floor_cells * dx])
        m = 0.5 * dx
        lo = np.array([c[0] - a + m, c[1] - a + m, c[2] - az + m])
        hi = np.array([c[0] + a - m, c[1] + a - m, c[2] - az + m + 0.1])
        x = _box_points(rng, n, lo, hi)
        v = np.zeros((n, 3))
        target = (c[0] + rng.uniform(-0.2, 0.2) * 0.25, c[1] + rng.uniform(-0.2, 0.2) * 0.25,
                  c[2] + rng.uniform(0.0, 0.3) * 0.25)
        spec = EnvSpec(n_particles=n, grid_res=G, substeps=substeps, dt=dt, material="fluid",
                       E=0.0, nu=0.0, rho=1e3, p_vol=float(np.prod(hi - lo)) / n, bulk=1e4, visc=1e-3,
                       collider="container", coll_dims=(a, w, az, 0.0), coll_mu=0.5, alpha=666.0,
                       act_map=(0, 1, 2), act_scale=(0.005, 0.005, 0.005), reward="reach",
                       n_sub=min(250, n), rparam=(float(target[0]), float(target[1]), float(target[2]), 0.0),
                       pose0=(float(c[0]), float(c[1]), float(c[2]), 0.0))
        specs.append(spec)
        inits.append(_rest_state(x, v))
        acts.append(rng.normal(0.0, action_std, (T, 3)))
    return Workload("fluid", specs, inits, _pad_actions(acts, T), T)


# ----------------------------------------------------------------------------- C4

def jumper(n_envs: int = 64, seed: int = 0, n: int = 100_000, G: int = 96, substeps: int = 20,
           T: int = 64, n_groups: int = 222) -> Workload:
    """Soft quadruped: torso 0.3 x 0.15 x 0.08 on four 0.06 x 0.06 x 0.1 legs.  Leg particles
    are neo-Hookean muscle with an active fibre stress scaled by per-group actions in
    [-1, 1] (n_groups groups by spatial binning); the rest is passive (E=3e4, nu=0.3)."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / G
    specs, inits, acts = [], [], []
    torso = np.array([0.3, 0.15, 0.08])
    leg = np.array([0.06, 0.06, 0.1])
    vol_t = float(np.prod(torso))
    vol_l = float(np.prod(leg))
    vol = vol_t + 4 * vol_l
    for e in range(n_envs):
        z0 = 3 * dx + 0.5 * dx + rng.uniform(0.0, 0.02)
        cx, cy = 0.5 + rng.uniform(-0.05, 0.05), 0.5 + rng.uniform(-0.05, 0.05)
        n_t = int(round(n * vol_t / vol))
        n_l = [(n - n_t) // 4 + (1 if i < (n - n_t) % 4 else 0) for i in range(4)]
        t_lo = np.array([cx - torso[0] / 2, cy - torso[1] / 2, z0 + leg[2]])
        xs = [_box_points(rng, n_t, t_lo, t_lo + torso)]
        gs = [np.full(n_t, -1, np.int32)]
        per_leg = (n_groups + 3) // 4
        for i, (sx, sy) in enumerate(((-1, -1), (1, -1), (-1, 1), (1, 1))):
            l_lo = np.array([cx + sx * (torso[0] / 2 - leg[0] / 2) - leg[0] / 2,
                             cy + sy * (torso[1] / 2 - leg[1] / 2) - leg[1] / 2, z0])
            p = _box_points(rng, n_l[i], l_lo, l_lo + leg)
            u = (p - l_lo) / leg
            b = (np.minimum((u[:, 2] * (per_leg // 4)).astype(int), per_leg // 4 - 1) * 4
                 + (u[:, 0] > 0.5).astype(int) * 2 + (u[:, 1] > 0.5).astype(int))
            g = np.minimum(i * per_leg + b, n_groups - 1).astype(np.int32)
            xs.append(p)
            gs.append(g)
        x = np.concatenate(xs)
        grp = np.concatenate(gs)
        order = rng.permutation(n)
        x, grp = x[order], grp[order]
        v = np.zeros((n, 3))
        init = _rest_state(x, v)
        init.group = np.ascontiguousarray(grp.astype(np.int32))
        spec = EnvSpec(n_particles=n, grid_res=G, substeps=substeps, dt=1e-4, material="muscle",
                       E=3e4, nu=0.3, rho=1e3, p_vol=vol / n, act_stress=1.5e4, n_groups=n_groups,
                       ground_mu=0.5, reward="jump", n_sub=min(250, n),
                       rparam=(float(z0 + leg[2] + torso[2] / 2), 3.0, 1e-4, 0.0))
        specs.append(spec)
        inits.append(init)
        acts.append(rng.uniform(-1.0, 1.0, (T, n_groups)))
    return Workload("jumper", specs, inits, _pad_actions(acts, T), T)


# ----------------------------------------------------------------------------- HandFlip-like

def handflip(n_envs: int = 128, seed: int = 0, n: int = 2500, G: int = 48, substeps: int = 40,
             T: int = 16, n_caps: int = 6, action_std: float = 0.5) -> Workload:
    """Elastoplastic slab (von Mises, E=4000, nu=0.2, sigma_y=130, rho=1) resting on a row of
    n_caps parallel capsule fingers (radius 0.015, half-length 0.1 along x, 0.035 apart in y)
    just above the floor; each finger is driven on its own by 4-DoF relative-pose actions
    (dx, dy, dz, dtheta_z) ~ N(0, 0.5), 4 n_caps actions per step (24 for six fingers), with
    dt=5e-5, 40 substeps, boundary friction 0.5 on a 48^3 grid.  The union of the capsules is
    a synthetic stand-in for the articulated hand, whose meshes are not available."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / G
    R, hl, gap = 0.015, 0.1, 0.035
    specs, inits, acts = [], [], []
    for e in range(n_envs):
        off = rng.uniform(-0.03, 0.03, 2)
        zf = 3 * dx + R + 0.37 * dx
        y0 = 0.5 + off[1] - 0.5 * (n_caps - 1) * gap
        size = np.array([0.14, max(0.1, (n_caps - 1) * gap), 0.04]) * rng.uniform(0.9, 1.1)
        lo = np.array([0.5 + off[0] - size[0] / 2, 0.5 + off[1] - size[1] / 2, zf + R + 0.5 * dx])
        hi = lo + size
        x = _box_points(rng, n, lo, hi)
        v = np.zeros((n, 3))
        spec = EnvSpec(n_particles=n, grid_res=G, substeps=substeps, dt=5e-5, material="vonmises",
                       E=4000.0, nu=0.2, rho=1.0, p_vol=float(np.prod(size)) / n, yield_stress=130.0,
                       c_y=2.0, collider="capsules", n_caps=n_caps, coll_dims=(R, hl, 0.0, 0.0),
                       cap_offset=(0.0, gap, 0.0), coll_mu=0.5, alpha=666.0,
                       act_scale=(0.005, 0.005, 0.005, 0.05), ground_mu=0.5, reward="none",
                       n_sub=min(250, n), pose0=(float(0.5 + off[0]), float(y0), float(zf), 0.0))
        specs.append(spec)
        inits.append(_rest_state(x, v))
        acts.append(rng.normal(0.0, action_std, (T, 4 * n_caps)))
    return Workload("handflip", specs, inits, _pad_actions(acts, T), T)


# ----------------------------------------------------------------------------- tet meshes

def voxel_mesh(occ, size, origin=(0.0, 0.0, 0.0)):
    """Tetrahedral mesh of the occupied voxels occ[i, j, k] (edge `size`): shared lattice
    vertices, five tetrahedra per voxel, the split mirrored on alternate voxels so that
    neighbouring faces carry the same diagonal.  Returns (rest (n_v, 3) float32, tets
    (n_t, 4) int32)."""
    occ = np.asarray(occ, bool)
    index = {}
    verts = []

    def vid(p):
        if p not in index:
            index[p] = len(verts)
            verts.append(p)
        return index[p]

    # corners (dx, dy, dz) of the five tetrahedra of a voxel; the fifth is the central one
    five = (((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)), ((1, 1, 0), (0, 1, 0), (1, 0, 0), (1, 1, 1)),
            ((1, 0, 1), (1, 0, 0), (0, 0, 1), (1, 1, 1)), ((0, 1, 1), (0, 0, 1), (0, 1, 0), (1, 1, 1)),
            ((1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1)))
    tets = []
    for i, j, k in zip(*np.nonzero(occ)):
        mirror = (i + j + k) % 2 == 1
        for tet in five:
            tets.append([vid((i + (1 - c[0] if mirror else c[0]), j + c[1], k + c[2])) for c in tet])
    rest = np.asarray(verts, np.float64) * size + np.asarray(origin, np.float64)
    return rest.astype(np.float32), np.asarray(tets, np.int32)


def softjumper(n_envs: int = 256, seed: int = 0, substeps: int = 80, T: int = 16, scale: float = 0.05,
               act_scale: float = 0.2) -> Workload:
    """SoftJumper (App. E) as tetrahedral FEM: a quadruped of voxels (a 7 x 4 x 2 torso on four
    2 x 2 x 2 legs, edge `scale`), 180 vertices and 440 elements, stable neo-Hookean with
    lambda = mu = 1000 (E = 2500, nu = 0.25), rho = 1, k_damp = 1, h = 1/60 in 80 substeps,
    ground z = 0 with friction 0.5.  Actions: one activation per pair of elements (220),
    U(-1, 1), scaled by act_scale into the elements' volume-ratio shift.  Reward: mean forward
    velocity + 3 (mean height - h0) - 1e-4 |a|^2 over all vertices.  Per env the body is
    scaled by U(0.9, 1.1) and offset by U(-0.08, 0.08) in x, y and U(0, 0.04) in z."""
    rng = np.random.default_rng(seed)
    occ = np.zeros((7, 4, 4), bool)
    occ[:, :, 2:4] = True
    for i0 in (0, 5):
        for j0 in (0, 2):
            occ[i0:i0 + 2, j0:j0 + 2, 0:2] = True
    rest0, tets = voxel_mesh(occ, 1.0)
    n_t = tets.shape[0]
    n_act = (n_t + 1) // 2
    group = (np.arange(n_t) // 2).astype(np.int32)
    specs, inits, acts = [], [], []
    for e in range(n_envs):
        sc = scale * rng.uniform(0.9, 1.1)
        off = np.array([rng.uniform(-0.08, 0.08), rng.uniform(-0.08, 0.08), rng.uniform(0.0, 0.04)])
        centre = np.array([0.5 - 3.5 * sc, 0.5 - 2.0 * sc, 0.0])
        rest = (rest0.astype(np.float64) * sc + centre + off).astype(np.float32)
        n = rest.shape[0]
        h0 = float(np.float32(rest[:, 2].astype(np.float64).mean()))
        spec = EnvSpec(n_particles=n, grid_res=8, substeps=substeps, dt=(1.0 / 60.0) / substeps, material="fem",
                       E=2500.0, nu=0.25, rho=1.0, act_stress=act_scale, n_groups=n_act, ground_mu=0.5,
                       reward="jump", n_sub=n, rparam=(h0, 3.0, 1e-4, 0.0), k_damp=1.0, ground_z=0.0,
                       fem_tets=tets, fem_rest=rest, fem_group=group, bound=0)
        specs.append(spec)
        inits.append(_rest_state(rest, np.zeros((n, 3))))
        acts.append(rng.uniform(-1.0, 1.0, (T, n_act)))
    return Workload("softjumper", specs, inits, _pad_actions(acts, T), T)
