"""Pins of the FP64 tetrahedral-FEM oracle (App. D.2 stable neo-Hookean elements, semi-implicit
Euler; App. E SoftJumper damping, activations and reward) against what the mathematics fixes:

- the stress is the energy's gradient, and its adjoint is the energy's Hessian (central
  differences);
- F = I is stress free (alpha = 1 + 3 mu / (4 lam)); an activation a gives P = -lam a I there;
- internal forces sum to zero and carry no torque (translation and rotation invariance of
  the energy), and equal -dE/dx;
- a rest mesh in free fall follows the closed form of the discrete scheme;
- the ground stops a falling vertex and applies Coulomb friction;
- the checkpointed reverse mode matches central differences of a rollout loss;
- a substep commutes with vertical-axis turns and horizontal shifts of the body;
- rest volumes, Dm^-1 and lumped masses of a voxel mesh in closed form.
"""
import numpy as np

from oracle import fem
from paper_2412_12089_gb300 import workloads as wl


def _mesh(n=(2, 1, 1), size=0.1, rng=None, jitter=0.0, **kw):
    occ = np.ones(n, bool)
    rest, tets = wl.voxel_mesh(occ, size, origin=(0.3, 0.3, 0.3))
    group = (np.arange(tets.shape[0]) % max(kw.get("n_act", 1), 1)).astype(np.int32)
    s = fem.spec(rest.shape[0], tets.shape[0], **kw)
    m = fem.Mesh(s, tets, group, rest, kw.get("rho", 1.0))
    x = rest.astype(np.float64)
    if rng is not None and jitter:
        x = x + jitter * rng.standard_normal(x.shape)
    return m, x


def _rand_F(rng, scale=0.3):
    while True:
        F = np.eye(3) + scale * rng.standard_normal((3, 3))
        if np.linalg.det(F) > 0.3:
            return F


def test_stress_is_energy_gradient():
    rng = np.random.default_rng(1)
    s = fem.spec(4, 1, mu=700.0, lam=1900.0)
    for _ in range(10):
        F, a = _rand_F(rng), rng.uniform(-0.3, 0.3)
        P = fem.stress(s, F, a)
        h = 1e-6
        fd = np.zeros((3, 3))
        for i in range(3):
            for j in range(3):
                E = np.zeros((3, 3))
                E[i, j] = h
                fd[i, j] = (fem.psi(s, F + E, a) - fem.psi(s, F - E, a)) / (2 * h)
        assert np.abs(fd - P).max() <= 1e-6 * np.abs(P).max()


def test_rest_is_stress_free_and_activation_closed_form():
    s = fem.spec(4, 1, mu=700.0, lam=1900.0)
    assert np.abs(fem.stress(s, np.eye(3), 0.0)).max() < 1e-12
    P = fem.stress(s, np.eye(3), 0.25)
    assert np.allclose(P, -1900.0 * 0.25 * np.eye(3), rtol=1e-13, atol=1e-10)
    # the energy is minimal at rest along any small deformation
    rng = np.random.default_rng(2)
    for _ in range(5):
        D = rng.standard_normal((3, 3))
        assert fem.psi(s, np.eye(3) + 1e-3 * D) > fem.psi(s, np.eye(3))


def test_stress_vjp_is_energy_hessian():
    rng = np.random.default_rng(3)
    s = fem.spec(4, 1, mu=800.0, lam=1200.0)
    for _ in range(10):
        F, a = _rand_F(rng), rng.uniform(-0.3, 0.3)
        Pb = rng.standard_normal((3, 3))
        Fb, ab = fem.stress_vjp(s, F, a, Pb)
        h = 1e-6
        for _ in range(3):
            D = rng.standard_normal((3, 3))
            fd = np.sum(Pb * (fem.stress(s, F + h * D, a) - fem.stress(s, F - h * D, a))) / (2 * h)
            assert abs(fd - np.sum(Fb * D)) <= 1e-6 * (abs(fd) + np.abs(Fb).max())
        fda = np.sum(Pb * (fem.stress(s, F, a + h) - fem.stress(s, F, a - h))) / (2 * h)
        assert abs(fda - ab) <= 1e-6 * (abs(fda) + 1.0)


def test_forces_balance_and_are_energy_gradient():
    rng = np.random.default_rng(4)
    m, x = _mesh((2, 2, 1), rng=rng, jitter=0.01, mu=1000.0, lam=1500.0, n_act=3)
    ae = rng.uniform(-0.2, 0.2, m.spec.n_t)
    f = fem.forces(m, x, np.zeros_like(x), ae)
    scale = np.abs(f).max()
    assert np.abs(f.sum(0)).max() <= 1e-12 * scale * len(f)
    torque = np.cross(x, f).sum(0)
    assert np.abs(torque).max() <= 1e-12 * scale * len(f)
    h = 1e-7
    for _ in range(6):
        i, k = rng.integers(0, len(x)), rng.integers(0, 3)
        xp, xm = x.copy(), x.copy()
        xp[i, k] += h
        xm[i, k] -= h
        fd = -(fem.energy(m, xp, ae) - fem.energy(m, xm, ae)) / (2 * h)
        assert abs(fd - f[i, k]) <= 1e-6 * scale, (i, k, fd, f[i, k])
    # damping forces of a velocity field also balance
    m2, _ = _mesh((2, 2, 1), rng=rng, mu=1000.0, lam=1500.0, k_damp=2.0)
    v = rng.standard_normal(x.shape)
    fd_ = fem.forces(m2, m2.rest_x, v) - fem.forces(m2, m2.rest_x, np.zeros_like(v))
    assert np.abs(fd_.sum(0)).max() <= 1e-12 * np.abs(fd_).max() * len(fd_)


def test_free_fall_closed_form():
    # dt well inside the explicit scheme's stability limit, so rounding does not grow
    m, x0 = _mesh((2, 1, 2), mu=1000.0, lam=1000.0, k_damp=1.0, dt=1e-4)
    g = np.array([0.0, 0.0, -9.8])
    v0 = np.tile([0.3, -0.2, 0.5], (len(x0), 1))
    x, v = x0.copy(), v0.copy()
    n = 25
    for _ in range(n):
        x, v, st = fem.substep(m, x, v)
        assert st == 0
    dt = 1e-4
    assert np.abs(v - (v0 + n * dt * g)).max() < 1e-12
    assert np.abs(x - (x0 + n * dt * v0 + dt * dt * g * n * (n + 1) / 2)).max() < 1e-12


def test_ground_stops_and_rubs():
    m, x0 = _mesh((1, 1, 1), mu=1000.0, lam=1000.0, dt=1e-3, ground_mu=0.4, gravity=(0.0, 0.0, 0.0))
    # the bottom face sits on the ground; a uniform velocity (no forces) down and sideways
    m.spec.ground_z = float(x0[:, 2].min())
    v0 = np.tile([0.5, 0.0, -0.2], (len(x0), 1))
    x, v, _ = fem.substep(m, x0, v0)
    bottom = x0[:, 2] <= m.spec.ground_z
    assert bottom.any() and (~bottom).any()
    assert np.all(v[bottom, 2] == 0.0)
    assert np.allclose(v[bottom, 0], 0.5 * (1.0 + 0.4 * (-0.2) / 0.5))
    assert np.allclose(v[~bottom], v0[~bottom])


def test_rollout_adjoint_matches_finite_differences():
    rng = np.random.default_rng(7)
    # two elements' worth of voxels, damping, activations in 3 groups, ground contact with
    # friction for the bottom vertices, jump reward
    m, x0 = _mesh((2, 1, 1), rng=rng, jitter=0.004, mu=600.0, lam=900.0, k_damp=0.5, dt=2e-4, S=3, n_act=3,
                  act_scale=0.2, ground_z=0.305, ground_mu=0.3, reward_kind=3, rparam=(0.3, 3.0, 1e-2, 0.0))
    v0 = 0.3 * rng.standard_normal(x0.shape)
    v0[:, 2] -= 0.5
    T = 2
    acts = rng.uniform(-1, 1, (T, 3))
    rbar = rng.standard_normal(T)
    xw, vw = rng.standard_normal(x0.shape), rng.standard_normal(x0.shape)

    def loss(x, v, a):
        xT, vT, r, _ = fem.rollout(m, x, v, a)
        return float((r * rbar).sum() + (xT * xw).sum() + (vT * vw).sum())

    ag, xb, vb, st = fem.rollout_adj(m, x0, v0, acts, xbT=xw, vbT=vw, rbar=rbar)
    assert np.abs(ag).max() > 0
    h = 1e-6
    for t in range(T):
        for j in range(3):
            ap, am = acts.copy(), acts.copy()
            ap[t, j] += h
            am[t, j] -= h
            fd = (loss(x0, v0, ap) - loss(x0, v0, am)) / (2 * h)
            assert abs(fd - ag[t, j]) <= 1e-5 * (abs(fd) + np.abs(ag).max() * 1e-2), (t, j, fd, ag[t, j])
    for arr, g, name in ((x0, xb, "x"), (v0, vb, "v")):
        for _ in range(6):
            i, k = rng.integers(0, len(arr)), rng.integers(0, 3)
            p, q = arr.copy(), arr.copy()
            p[i, k] += h
            q[i, k] -= h
            args_p = (p, v0) if name == "x" else (x0, p)
            args_q = (q, v0) if name == "x" else (x0, q)
            fd = (loss(*args_p, acts) - loss(*args_q, acts)) / (2 * h)
            assert abs(fd - g[i, k]) <= 1e-5 * (abs(fd) + np.abs(g).max() * 1e-2), (name, i, k, fd, g[i, k])


def test_softjumper_mesh_and_rollout():
    w = wl.softjumper(n_envs=1, seed=3, T=2, substeps=80)
    s = w.specs[0]
    assert s.n_particles == 180 and s.fem_tets.shape == (440, 4) and s.n_groups == 220
    m = fem.make_mesh(s)
    assert np.all(m.vol > 0) and np.isclose(m.vol.sum(), (56 + 32) * (np.linalg.det(
        np.diag(s.fem_rest.max(0) - s.fem_rest.min(0))) / (7 * 4 * 4)), rtol=1e-5)
    x, v, r, st = fem.rollout(m, w.inits[0].x, w.inits[0].v, w.actions[:2, 0, :220])
    assert st == 0 and np.all(np.isfinite(x)) and x[:, 2].min() > -0.01


def test_substep_commutes_with_vertical_rotations_and_horizontal_shifts():
    """Objectivity of the semi-implicit step: turning the deformed, moving body about a
    vertical axis (rest shape unchanged) turns the result, and shifting it horizontally shifts
    the result.  Gravity, the ground and its friction are vertical or horizontal-isotropic, the
    energy and the damping stress k_damp * Fdot are frame-indifferent, and the activations
    act on J.  A dropped or transposed term in P or in the corner forces breaks this."""
    rng = np.random.default_rng(31)
    m, x = _mesh((2, 2, 1), rng=rng, jitter=0.001, mu=900.0, lam=1300.0, k_damp=1.5, n_act=3, ground_mu=0.4,
                 act_scale=0.3, dt=1e-4)
    m.spec.ground_z = float(np.sort(x[:, 2])[3])  # four vertices at or below the ground
    v = 0.3 * rng.standard_normal(x.shape)
    v[:, 2] = -0.2 - np.abs(v[:, 2])  # moving down: the ground projects and rubs
    ae = rng.uniform(-0.2, 0.2, m.spec.n_t)
    x1, v1, st = fem.substep(m, x, v, ae)
    on = x[:, 2] <= m.spec.ground_z
    assert st == 0 and on.sum() >= 4 and np.all(v1[on, 2] == 0.0)
    assert (np.hypot(v1[on, 0], v1[on, 1]) > 0.0).sum() >= 2  # sliding: friction depends on direction
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0.0], [np.sin(th), np.cos(th), 0.0], [0.0, 0.0, 1.0]])
    p = np.array([0.4, 0.35, 0.0])  # a point on the axis
    xr, vr, st = fem.substep(m, (x - p) @ R.T + p, v @ R.T, ae)
    assert st == 0
    assert np.abs(xr - ((x1 - p) @ R.T + p)).max() <= 1e-13
    assert np.abs(vr - v1 @ R.T).max() <= 1e-11 * np.abs(v1).max()
    s = np.array([0.125, -0.0625, 0.0])
    xs, vs, st = fem.substep(m, x + s, v, ae)
    assert st == 0
    assert np.abs(xs - (x1 + s)).max() <= 1e-13 and np.abs(vs - v1).max() <= 1e-11 * np.abs(v1).max()
    assert np.abs(v1 - v).max() > 1e-4  # the step changed the state


def test_rest_quantities_closed_form():
    """Rest data of a voxel mesh: the five elements of each voxel fill it (their rest volumes
    sum to the voxel count times edge^3, the central element holding a third of each voxel),
    Dm^-1 inverts each element's edge matrix, and the lumped masses rho V / 4 per corner add
    up to the body's mass."""
    m, x = _mesh((3, 2, 2), size=0.05, rho=7.0)
    n_vox, size = 12, 0.05
    # the lattice is stored in FP32, so the voxels are cubes to about 1e-7
    assert abs(m.vol.sum() - n_vox * size ** 3) <= 1e-6 * n_vox * size ** 3
    central = m.vol.reshape(n_vox, 5)[:, 4]
    assert np.allclose(central, size ** 3 / 3.0, rtol=1e-6)
    for e, t in enumerate(m.tets):
        Dm = np.stack([x[t[c + 1]] - x[t[0]] for c in range(3)], 1)
        assert np.allclose(m.dminv[e].reshape(3, 3) @ Dm, np.eye(3), atol=1e-10)
        assert abs(abs(np.linalg.det(Dm)) / 6.0 - m.vol[e]) <= 1e-15
    assert abs((1.0 / m.inv_mass).sum() - 7.0 * m.vol.sum()) <= 1e-12 * 7.0 * m.vol.sum()
