"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

The oracle (oracle/) is the reference every CUDA parity test compares with, so it is
itself checked here against things other than itself: properties of quadratic
B-splines, conservation laws of the MLS-MPM transfers, the closed-form discrete free
fall, closed-form stresses, return-mapping invariants, numpy's SVD, analytic SDFs,
central finite differences of its own forward pass and a dot-product test of its
reverse pass.  Each test names the passage of arXiv 2412.12089 it pins.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2412_12089_gb300 import workloads as wl

RNG = np.random.default_rng(1234)


def spec_for(material="neohookean", G=8, dt=1e-4, **kw):
    base = dict(n_particles=1, grid_res=G, substeps=1, dt=dt, material=material, E=1e4, nu=0.3, rho=1e3,
                p_vol=1e-6, yield_stress=50.0, c_y=2.0, bulk=1e4, visc=1e-3, act_stress=1.5e4, n_groups=4)
    base.update(kw)
    return orc.make_spec(wl.EnvSpec(**base))


def rand_rot(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


# ------------------------------------------------------------------ B-spline weights (App. D.3, MLS-MPM)

def test_weights_moments():
    """Quadratic B-spline: partition of unity, zero first moment, second moment 1/4
    (this is what makes D^-1 = 4/dx^2); derivatives match finite differences."""
    for fx in np.linspace(0.5, 1.4999, 37):
        w, dw = orc.weights(fx)
        r = np.arange(3) - fx
        assert abs(w.sum() - 1) < 1e-14
        assert abs((w * r).sum()) < 1e-14
        assert abs((w * r * r).sum() - 0.25) < 1e-14
        h = 1e-7
        wp, _ = orc.weights(fx + h)
        wm, _ = orc.weights(fx - h)
        assert np.allclose((wp - wm) / (2 * h), dw, atol=1e-7)


# ------------------------------------------------------------------ transfers

def _rand_state(n, G, rng, lo=0.35, hi=0.65, Fs=0.05, Cs=0.5, vs=0.3):
    x = lo + (hi - lo) * rng.random((n, 3))
    v = vs * rng.standard_normal((n, 3))
    C = Cs * rng.standard_normal((n, 3, 3))
    F = np.eye(3) + Fs * rng.standard_normal((n, 3, 3))
    return orc.State(x, v, C, F)


@pytest.mark.parametrize("material", ["neohookean", "vonmises", "fluid"])
def test_p2g_conservation(material):
    """P2G (App. D.3 CPIC step 2): grid mass = particle mass; grid momentum = particle
    momentum (the affine and stress terms cancel because sum_i w r = 0); grid angular
    momentum = sum m x x v + m (dx^2/4) eps:C^T (APIC; the symmetric stress adds none)."""
    sp = spec_for(material, G=16)
    st = _rand_state(64, 16, RNG)
    g, status = orc.p2g(sp, st)
    assert status == 0
    G = 16
    assert abs(g[..., 0].sum() - 64 * sp.p_mass) < 1e-13 * 64 * sp.p_mass
    pm = sp.p_mass * st.v.sum(0)
    assert np.allclose(g[..., 1:].sum((0, 1, 2)), pm, rtol=1e-12, atol=1e-14)
    iz, iy, ix = np.meshgrid(np.arange(G), np.arange(G), np.arange(G), indexing="ij")
    xi = np.stack([ix, iy, iz], -1) / G
    Lg = np.cross(xi, g[..., 1:]).sum((0, 1, 2))
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1
    dx = 1.0 / G
    Lp = (sp.p_mass * np.cross(st.x, st.v)).sum(0)
    Lp += sp.p_mass * dx * dx / 4 * np.einsum("kab,pba->k", eps, st.C)
    assert np.allclose(Lg, Lp, rtol=1e-10, atol=1e-15)


def test_g2p_affine_reproduction():
    """G2P (CPIC step 4) with quadratic B-splines reproduces an affine grid velocity
    field exactly: v_p = a + B x_p and C_p = B (pins D^-1 = 4/dx^2 and r = x_i - x_p)."""
    G = 16
    sp = spec_for("neohookean", G=G, dt=1e-3)
    st = _rand_state(40, G, RNG)
    a = RNG.standard_normal(3)
    B = RNG.standard_normal((3, 3))
    iz, iy, ix = np.meshgrid(np.arange(G), np.arange(G), np.arange(G), indexing="ij")
    xi = np.stack([ix, iy, iz], -1) / G
    gv = a + xi @ B.T
    out, status = orc.g2p(sp, st, gv)
    vp = a + st.x @ B.T
    assert np.allclose(out.v, vp, atol=1e-12)
    assert np.allclose(out.C, np.broadcast_to(B, out.C.shape), atol=1e-10)
    assert np.allclose(out.x, st.x + sp.dt * vp, atol=1e-14)
    Fexp = np.einsum("ij,pjk->pik", np.eye(3) + sp.dt * B, st.F)
    assert np.allclose(out.F, Fexp, atol=1e-12)


def test_g2p_momentum_matches_grid():
    """P2G followed directly by G2P (no forces, no walls) conserves linear momentum,
    sum m v_p' = sum_i m_i v_i, and APIC angular momentum at the pre-advection positions,
    sum m (x_p x v_p' + (dx^2/4) eps:C_p'^T) = sum_i m_i x_i x v_i, for any grid field
    (C_p' = D^-1 sum w v_i r^T makes the particles' spin carry the stencil's moment)."""
    G = 16
    sp = spec_for("neohookean", G=G, bound=0, gravity=(0.0, 0.0, 0.0))
    st = _rand_state(50, G, RNG)
    st.F[:] = np.eye(3)
    g, _ = orc.p2g(sp, st)
    gv = orc.grid_update(sp, g)
    m = g[..., 0]
    out, _ = orc.g2p(sp, st, gv)
    assert np.allclose((sp.p_mass * out.v).sum(0), (m[..., None] * gv).sum((0, 1, 2)), rtol=1e-11, atol=1e-15)
    assert np.allclose((m[..., None] * gv).sum((0, 1, 2)), sp.p_mass * st.v.sum(0), rtol=1e-11, atol=1e-15)
    # a non-affine grid field (random per node) on the same masses
    gr = RNG.standard_normal(gv.shape)
    out, _ = orc.g2p(sp, st, gr)
    iz, iy, ix = np.meshgrid(np.arange(G), np.arange(G), np.arange(G), indexing="ij")
    xi = np.stack([ix, iy, iz], -1) / G
    Lg = (m[..., None] * np.cross(xi, gr)).sum((0, 1, 2))
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1
    Lp = (sp.p_mass * np.cross(st.x, out.v)).sum(0)
    Lp += sp.p_mass / (4 * G * G) * np.einsum("kab,pba->k", eps, out.C)
    assert np.allclose(Lp, Lg, rtol=1e-11, atol=1e-15)


def test_free_fall_closed_form():
    """Undeformed block, uniform v0, gravity only, far from walls: after k substeps of the
    discrete scheme v = v0 + k dt g, x = x0 + k dt v0 + dt^2 g k(k+1)/2, C = 0, F = I."""
    w = wl.cube(seed=3, n=300, G=16, substeps=12)
    es = w.specs[0]
    sp = orc.make_spec(es)
    init = w.inits[0]
    v0 = np.array([0.05, -0.02, 0.1])
    st = orc.State(init.x, np.broadcast_to(v0, init.v.shape), init.C, init.F)
    out, q, rew, status = orc.rollout(sp, st, np.zeros(4), np.zeros((1, 1)))
    k, dt = es.substeps, es.dt
    g = np.array(es.gravity)
    assert np.allclose(out.v, v0 + k * dt * g, atol=1e-12)
    assert np.allclose(out.x, st.x + k * dt * v0 + dt * dt * g * k * (k + 1) / 2, atol=1e-13)
    assert np.abs(out.C).max() < 1e-10
    assert np.abs(out.F - np.eye(3)).max() < 1e-12


# ------------------------------------------------------------------ constitutive laws (App. D.3)

@pytest.mark.parametrize("material", ["neohookean", "vonmises", "fluid", "muscle"])
def test_zero_stress_at_identity(material):
    sp = spec_for(material)
    assert np.abs(orc.tau(sp, np.eye(3))).max() < 1e-12


@pytest.mark.parametrize("material", ["neohookean", "vonmises"])
def test_small_strain_limit(material):
    """tau(I + eta S) = 2 mu eta S + lam eta tr(S) I + O(eta^2) (linear elasticity)."""
    sp = spec_for(material)
    S = RNG.standard_normal((3, 3))
    S = 0.5 * (S + S.T)
    eta = 1e-6
    t = orc.tau(sp, np.eye(3) + eta * S)
    lin = 2 * sp.mu * eta * S + sp.lam * eta * np.trace(S) * np.eye(3)
    assert np.abs(t - lin).max() < 1e-4 * np.abs(lin).max()


def test_hencky_closed_form():
    """App. D.3 elastic law: for F = R diag(s) Q^T, tau = R diag(2 mu log s + lam sum log s) R^T."""
    sp = spec_for("vonmises")
    for _ in range(5):
        s = RNG.uniform(0.7, 1.3, 3)
        R, Q = rand_rot(RNG), rand_rot(RNG)
        F = R @ np.diag(s) @ Q.T
        t = 2 * sp.mu * np.log(s) + sp.lam * np.log(s).sum()
        assert np.allclose(orc.tau(sp, F), R @ np.diag(t) @ R.T, atol=1e-9 * np.abs(t).max())


def test_neohookean_closed_form():
    sp = spec_for("neohookean")
    F = np.diag([1.1, 0.9, 1.05])
    J = np.prod(np.diag(F))
    exp = sp.mu * (F @ F.T - np.eye(3)) + sp.lam * np.log(J) * np.eye(3)
    assert np.allclose(orc.tau(sp, F), exp, atol=1e-9)


def test_muscle_fibre_stress():
    """Active fibre stress a * s * (F e_z)(F e_z)^T on top of the neo-Hookean part."""
    sp = spec_for("muscle")
    nh = spec_for("neohookean")
    F = np.eye(3) + 0.1 * RNG.standard_normal((3, 3))
    f = F[:, 2]
    assert np.allclose(orc.tau(sp, F, a_g=0.7) - orc.tau(nh, F), 0.7 * sp.act_stress * np.outer(f, f), atol=1e-8)


def test_fluid_viscosity_rigid_rotation_and_dissipation():
    """The viscous part of the fluid stress is Newtonian: a rigid rotation (antisymmetric
    velocity gradient C) produces no viscous stress, and in any flow the viscous stress does
    non-negative work on the velocity gradient (tau_visc : C >= 0), equal to 2 visc J |sym C|^2.
    Checked on the stress the oracle returns with the bulk part taken out at the same J."""
    sp = spec_for("fluid")
    for J in (0.95, 1.0, 1.03):
        F = np.cbrt(J) * np.eye(3)
        base = orc.tau(sp, F, np.zeros((3, 3)))
        for _ in range(5):
            W = RNG.standard_normal((3, 3))
            W = W - W.T  # antisymmetric: a rigid rotation rate
            assert np.abs(orc.tau(sp, F, W) - base).max() < 1e-12 * max(1.0, np.abs(base).max())
            C = RNG.standard_normal((3, 3))
            tv = orc.tau(sp, F, C) - base
            work = float(np.sum(tv * C))
            assert work >= 0.0
            S = 0.5 * (C + C.T)
            assert abs(work - 2.0 * sp.visc * J * float(np.sum(S * S))) <= 1e-12 * max(1.0, abs(work))
            # a pure shear rate of the same magnitude but opposite sense dissipates equally
            assert abs(float(np.sum((orc.tau(sp, F, -C) - base) * -C)) - work) <= 1e-12 * max(1.0, work)


def test_fluid_closed_form():
    """App. D.3 fluid: P = K J (J-1) F^-T gives tau = K J (J-1) I; viscosity adds
    visc J (C + C^T)."""
    sp = spec_for("fluid")
    J = 0.97
    F = np.cbrt(J) * np.eye(3)
    C = RNG.standard_normal((3, 3))
    exp = sp.bulk * J * (J - 1) * np.eye(3) + sp.visc * J * (C + C.T)
    assert np.allclose(orc.tau(sp, F, C), exp, rtol=1e-12, atol=1e-12)


def test_return_mapping_invariants():
    """App. D.3 von Mises projection: after yielding |eps^_new| = c_y sigma_y / (2 mu),
    tr(eps) (so det F) is unchanged, the rotations are kept; below yield F is unchanged."""
    sp = spec_for("vonmises")
    target = sp.c_y * sp.yield_stress / (2 * sp.mu)
    for _ in range(5):
        s = RNG.uniform(0.85, 1.15, 3)
        R, Q = rand_rot(RNG), rand_rot(RNG)
        F = R @ np.diag(s) @ Q.T
        Fo = orc.project(sp, F)
        e = np.log(s)
        eh = e - e.mean()
        if np.linalg.norm(eh) <= target:
            assert np.allclose(Fo, F)
            continue
        so = np.linalg.svd(Fo, compute_uv=False)
        eo = np.log(so)
        assert abs(np.linalg.norm(eo - eo.mean()) - target) < 1e-10
        assert abs(np.linalg.det(Fo) - np.linalg.det(F)) < 1e-10
        en = e.mean() + target * eh / np.linalg.norm(eh)
        assert np.allclose(Fo, R @ np.diag(np.exp(en)) @ Q.T, atol=1e-10)
    F = np.eye(3) + 1e-4 * np.diag([1, -1, 0.5])
    assert np.allclose(orc.project(sp, F), F)


def test_fluid_projection():
    sp = spec_for("fluid")
    F = np.eye(3) + 0.1 * RNG.standard_normal((3, 3))
    Fo = orc.project(sp, F)
    J = np.linalg.det(F)
    assert np.allclose(Fo, np.cbrt(J) * np.eye(3))
    assert abs(np.linalg.det(Fo) - J) < 1e-12


# ------------------------------------------------------------------ SVD

@pytest.mark.parametrize("case", ["random", "identity", "aab", "reflection", "rank2", "scaled_rot"])
def test_svd(case):
    """F = U diag(s) V^T with det U = det V = +1; |s| equal numpy's singular values."""
    if case == "random":
        F = RNG.standard_normal((3, 3))
    elif case == "identity":
        F = np.eye(3)
    elif case == "aab":
        R, Q = rand_rot(RNG), rand_rot(RNG)
        F = R @ np.diag([1.2, 1.2, 0.8]) @ Q.T
    elif case == "reflection":
        F = np.diag([1.0, 0.9, -0.8])
    elif case == "rank2":
        F = RNG.standard_normal((3, 2)) @ RNG.standard_normal((2, 3))
    else:
        F = 1.7 * rand_rot(RNG)
    U, s, V = orc.svd3(F)
    assert np.abs(U @ np.diag(s) @ V.T - F).max() < 1e-13 * max(1, np.abs(F).max())
    assert np.abs(U.T @ U - np.eye(3)).max() < 1e-13
    assert np.abs(V.T @ V - np.eye(3)).max() < 1e-13
    assert abs(np.linalg.det(U) - 1) < 1e-12 and abs(np.linalg.det(V) - 1) < 1e-12
    assert np.allclose(np.abs(s), np.linalg.svd(F, compute_uv=False), atol=1e-13)
    assert np.all(np.diff(np.abs(s)) <= 1e-15)
    assert np.sign(s[2]) == np.sign(np.linalg.det(F)) or abs(s[2]) < 1e-12


# ------------------------------------------------------------------ colliders (App. D.3 softened contact)

def test_capsule_sdf_closed_form():
    sp = spec_for(collider="capsule", coll_dims=(0.03, 0.12, 0, 0))
    q = np.array([0.5, 0.5, 0.3, 0.0])
    d, n, H, vb = orc.collider(sp, [0.55, 0.5, 0.4], q)
    assert abs(d - (0.1 - 0.03)) < 1e-14 and np.allclose(n, [0, 0, 1])
    d, n, H, vb = orc.collider(sp, [0.5 + 0.12 + 0.05, 0.5, 0.3], q)
    assert abs(d - 0.02) < 1e-14 and np.allclose(n, [1, 0, 0])
    qr = np.array([0.5, 0.5, 0.3, np.pi / 2])  # yaw 90 deg: axis along y
    d, n, H, vb = orc.collider(sp, [0.5, 0.5 + 0.1, 0.3], qr)
    assert abs(d + 0.03) < 1e-14
    d, n, H, vb = orc.collider(sp, [0.6, 0.5, 0.3], qr, u=(1.0, 2.0, 3.0, 0.5))
    assert abs(d - 0.07) < 1e-12 and np.allclose(n, [1, 0, 0], atol=1e-12)
    assert np.allclose(vb, [1.0 - 0.5 * 0.0, 2.0 + 0.5 * 0.1, 3.0])


def test_box_and_container_sdf_closed_form():
    sp = spec_for(collider="box", coll_dims=(0.1, 0.2, 0.05, 0))
    q = np.array([0.5, 0.5, 0.5, 0.0])
    d, n, _, _ = orc.collider(sp, [0.5, 0.5, 0.5 + 0.05 + 0.01], q)
    assert abs(d - 0.01) < 1e-14 and np.allclose(n, [0, 0, 1])
    d, n, _, _ = orc.collider(sp, [0.5 + 0.1 + 0.03, 0.5 + 0.2 + 0.04, 0.5], q)
    assert abs(d - 0.05) < 1e-14 and np.allclose(n, [0.6, 0.8, 0])
    d, n, _, _ = orc.collider(sp, [0.52, 0.5, 0.5], q)
    assert abs(d + 0.05 - 0.0) < 1e-14 and np.allclose(n, [0, 0, 1]) or abs(d + 0.05) < 1e-14
    sc = spec_for(collider="container", coll_dims=(0.1, 0.02, 0.1, 0))
    q = np.array([0.5, 0.5, 0.3, 0.0])
    d, n, _, _ = orc.collider(sc, [0.5, 0.5, 0.3 - 0.1 + 0.004], q)  # above the floor
    assert abs(d - 0.004) < 1e-14 and np.allclose(n, [0, 0, 1])
    d, n, _, _ = orc.collider(sc, [0.5 + 0.1 - 0.003, 0.5, 0.3], q)  # next to +x wall
    assert abs(d - 0.003) < 1e-14 and np.allclose(n, [-1, 0, 0])


def test_container_nearest_box_and_ties():
    """The container is the union of a floor and four walls: its SDF is the smallest of the
    five box distances, and a point exactly as near to two boxes takes the first of them
    (floor, +x, -x, +y, -y), the rule both sides share.  Dyadic dimensions make the ties exact."""
    a, w, az = 0.125, 0.03125, 0.125
    sc = spec_for(collider="container", coll_dims=(a, w, az, 0))
    q = np.array([0.5, 0.5, 0.25, 0.0])
    e = 2.0 ** -7
    # inside the cavity, e from the floor's top face and e from the +x wall's inner face
    d, n, _, _ = orc.collider(sc, [0.5 + a - e, 0.5, 0.25 - az + e], q)
    assert d == e and np.array_equal(n, [0.0, 0.0, 1.0])
    # e from the -y wall and the +x wall at once: +x comes first
    d, n, _, _ = orc.collider(sc, [0.5 + a - e, 0.5 - a + e, 0.25], q)
    assert d == e and np.array_equal(n, [-1.0, 0.0, 0.0])
    # nearer to the -y wall than to the +x wall: the nearest box wins whatever its order
    d, n, _, _ = orc.collider(sc, [0.5 + a - 2 * e, 0.5 - a + e, 0.25], q)
    assert d == e and np.array_equal(n, [0.0, 1.0, 0.0])
    # inside the floor slab, nearer its top face than any wall: negative distance, up normal
    d, n, _, _ = orc.collider(sc, [0.5, 0.5, 0.25 - az - e], q)
    assert d == -e and np.array_equal(n, [0.0, 0.0, 1.0])


@pytest.mark.parametrize("kind,dims", [("capsule", (0.03, 0.12, 0, 0)), ("box", (0.08, 0.05, 0.04, 0)),
                                       ("container", (0.1, 0.02, 0.1, 0))])
def test_sdf_gradient_and_hessian_fd(kind, dims):
    """n = grad d and H = grad n by central differences, and the pose derivatives the
    adjoint uses: d/dc = -n, d/dtheta through the rotated frame."""
    sp = spec_for(collider=kind, coll_dims=dims)
    q = np.array([0.5, 0.52, 0.4, 0.3])
    h = 1e-7
    for _ in range(20):
        x = q[:3] + RNG.uniform(-0.15, 0.15, 3)
        d, n, H, _ = orc.collider(sp, x, q)
        gd = np.zeros(3)
        Hn = np.zeros((3, 3))
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            dp, np_, _, _ = orc.collider(sp, x + e, q)
            dm, nm, _, _ = orc.collider(sp, x - e, q)
            gd[k] = (dp - dm) / (2 * h)
            Hn[:, k] = (np_ - nm) / (2 * h)
        if np.abs(gd - n).max() > 1e-5:  # straddles a kink of the SDF (medial axis)
            continue
        assert np.allclose(gd, n, atol=1e-6)
        assert np.allclose(Hn, H, atol=1e-3 * max(1, np.abs(H).max()))


def test_contact_projection_closed_form():
    """Grid node deep inside the collider (s = 1): with mu_b = 0 the normal velocity into
    the body is removed; with a large mu_b the node sticks to the body; outside the body the
    blend is s = exp(-alpha d)."""
    G = 16
    for mu, expect in [(0.0, "slip"), (100.0, "stick")]:
        sp = spec_for(collider="box", coll_dims=(0.2, 0.2, 0.05, 0), coll_mu=mu, G=G, bound=0,
                      gravity=(0.0, 0.0, 0.0))
        g = np.zeros((G, G, G, 4))
        iz, iy, ix = 8, 8, 8
        g[iz, iy, ix] = [2.0, 2.0 * 0.3, 2.0 * 0.1, 2.0 * -0.5]
        q = np.array([0.5, 0.5, 0.5 + 0.01, 0.0])  # node 0.01 below the box top face
        gv = orc.grid_update(sp, g, q)
        v = gv[iz, iy, ix]
        if expect == "slip":
            # nearest face is the bottom face (n = -z): vn = +0.5 > 0 separating -> unchanged
            assert np.allclose(v, [0.3, 0.1, -0.5])
        q = np.array([0.5, 0.5, 0.5 - 0.04, 0.0])  # nearest face the top (n = +z), vn = -0.5
        v = orc.grid_update(sp, g, q)[iz, iy, ix]
        if expect == "slip":
            assert np.allclose(v, [0.3, 0.1, 0.0])
        else:
            assert np.allclose(v, [0.0, 0.0, 0.0])
    sp = spec_for(collider="box", coll_dims=(0.2, 0.2, 0.05, 0), coll_mu=0.0, G=G, bound=0, gravity=(0.0, 0.0, 0.0),
                  alpha=100.0)
    g = np.zeros((G, G, G, 4))
    g[8, 8, 8] = [1.0, 0.0, 0.0, -1.0]
    q = np.array([0.5, 0.5, 0.5 - 0.05 - 0.02, 0.0])  # node 0.02 above the top face
    v = orc.grid_update(sp, g, q)[8, 8, 8]
    s = np.exp(-100.0 * 0.02)
    assert np.allclose(v, [0, 0, -1.0 + s * 1.0])


def test_domain_walls():
    """Separating slip walls b nodes thick; the bottom wall applies Coulomb friction."""
    G = 16
    sp = spec_for(G=G, bound=3, gravity=(0.0, 0.0, 0.0), ground_mu=0.5)
    g = np.zeros((G, G, G, 4))
    g[1, 8, 8] = [1.0, 0.4, 0.3, -0.2]  # bottom layer, moving down
    g[8, 8, 14] = [1.0, 0.7, 0.1, 0.2]  # +x wall, moving out
    g[8, 1, 8] = [1.0, 0.2, 0.3, 0.1]  # -y wall, moving in (kept)
    gv = orc.grid_update(sp, g)
    L = np.hypot(0.4, 0.3)
    f = 1 + 0.5 * -0.2 / L
    assert np.allclose(gv[1, 8, 8], [0.4 * f, 0.3 * f, 0.0])
    assert np.allclose(gv[8, 8, 14], [0.0, 0.1, 0.2])
    assert np.allclose(gv[8, 1, 8], [0.2, 0.3, 0.1])


# ------------------------------------------------------------------ reverse mode vs central differences

def _fd_vjp(f, x, w, h):
    """Directional central differences <w, J e_k> for all k (x flattened)."""
    g = np.zeros(x.size)
    xf = x.reshape(-1)
    for k in range(x.size):
        xp = xf.copy()
        xp[k] += h
        xm = xf.copy()
        xm[k] -= h
        g[k] = ((f(xp.reshape(x.shape)) - f(xm.reshape(x.shape))) * w).sum() / (2 * h)
    return g.reshape(x.shape)


@pytest.mark.parametrize("material", ["neohookean", "muscle", "vonmises_yield", "fluid"])
def test_material_vjp_fd(material):
    mat = "vonmises" if material.startswith("vonmises") else material
    kw = {"yield_stress": 5.0} if material == "vonmises_yield" else {}
    sp = spec_for(mat, **kw)
    for F in [np.eye(3) + 0.08 * RNG.standard_normal((3, 3)), np.eye(3), np.eye(3) + 1e-9 * RNG.standard_normal((3, 3)),
              np.diag([1.05, 1.05, 0.97])]:
        C = 0.3 * RNG.standard_normal((3, 3))
        a = 0.6
        tb = RNG.standard_normal((3, 3))
        Fb, Cb, ab = orc.tau_vjp(sp, F, C, a, tb)
        scale = np.abs(Fb).max() + 1e-3 * (sp.mu + sp.lam + sp.bulk)
        fd = _fd_vjp(lambda Z: orc.tau(sp, Z, C, a), F, tb, 1e-6)
        assert np.abs(fd - Fb).max() < 1e-5 * scale, (material, F)
        fdc = _fd_vjp(lambda Z: orc.tau(sp, F, Z, a), C, tb, 1e-6)
        floor = 1e-14 * np.abs(orc.tau(sp, F, C, a)).max() * np.abs(tb).sum() / 1e-6  # FD rounding floor
        assert np.abs(fdc - Cb).max() < 1e-5 * (np.abs(Cb).max() + 1e-9) + floor
        if material == "muscle":
            fda = ((orc.tau(sp, F, C, a + 1e-6) - orc.tau(sp, F, C, a - 1e-6)) * tb).sum() / 2e-6
            assert abs(fda - ab) < 1e-6 * max(1, abs(ab))
        P = orc.project(sp, F + 0.02 * np.diag([1, -1, 0.3]))
        Ft = F + 0.02 * np.diag([1, -1, 0.3])
        Pb = RNG.standard_normal((3, 3))
        fdp = _fd_vjp(lambda Z: orc.project(sp, Z), Ft, Pb, 1e-7)
        assert np.abs(fdp - orc.project_vjp(sp, Ft, Pb)).max() < 1e-5 * max(1, np.abs(fdp).max()), material
        assert P.shape == (3, 3)


def test_return_mapping_vjp_degenerate():
    """Return-mapping adjoint where two singular values coincide (the divided difference
    takes its limit) while the projection is active."""
    sp = spec_for("vonmises", yield_stress=1.0)
    R, Q = rand_rot(RNG), rand_rot(RNG)
    Ft = R @ np.diag([1.1, 1.1, 0.9]) @ Q.T
    Pb = RNG.standard_normal((3, 3))
    fd = _fd_vjp(lambda Z: orc.project(sp, Z), Ft, Pb, 1e-7)
    assert np.abs(fd - orc.project_vjp(sp, Ft, Pb)).max() < 1e-5 * np.abs(fd).max()


CASES = {
    "nh": dict(material="neohookean"),
    "muscle": dict(material="muscle"),
    "vonmises": dict(material="vonmises", yield_stress=3.0),
    "fluid": dict(material="fluid"),
    "capsule": dict(material="neohookean", collider="capsule", coll_dims=(0.08, 0.1, 0, 0), coll_mu=0.4,
                    alpha=40.0),
    "box_ground": dict(material="vonmises", yield_stress=3.0, collider="box", coll_dims=(0.1, 0.06, 0.05, 0),
                       coll_mu=0.3, alpha=30.0, ground_mu=0.4),
    "container": dict(material="fluid", collider="container", coll_dims=(0.1, 0.05, 0.1, 0), coll_mu=0.5,
                      alpha=20.0),
}


def _tiny_case(name, seed, n=12, G=8):
    rng = np.random.default_rng(seed)
    kw = dict(CASES[name])
    sp = spec_for(G=G, dt=2e-3, bound=2, **kw)
    st = _rand_state(n, G, rng, lo=0.3, hi=0.7, vs=0.5)
    if name in ("container",):
        st.F = np.broadcast_to(np.eye(3), st.F.shape) * np.cbrt(1 + 0.02 * rng.standard_normal((n, 1, 1)))
    st.group = rng.integers(-1, 4, n).astype(np.int32)
    q = np.array([0.5, 0.5, 0.35, 0.2]) + 0.02 * rng.standard_normal(4)
    u = 0.3 * rng.standard_normal(4)
    act = np.concatenate([np.zeros(len(kw.get("act_map", ()))), rng.uniform(-1, 1, 4)])
    return sp, st, q, u, act


@pytest.mark.parametrize("name", list(CASES))
def test_substep_adjoint_fd(name):
    """Hand-derived reverse of one substep (G2P, grid, P2G adjoints) against central
    finite differences of the FP64 forward, for every input: state, collider pose and
    velocity, muscle actions."""
    sp, st, q, u, act = _tiny_case(name, seed=7)
    rng = np.random.default_rng(11)
    wts = [rng.standard_normal(a.shape) for a in st.arrays()]

    def loss(s, qq=q, uu=u, aa=act):
        o, _ = orc.substep(sp, s, qq, uu, aa)
        return sum((a * b).sum() for a, b in zip(o.arrays(), wts))

    adj, qb, ub, ab = orc.substep_adj(sp, st, wts, q, u, act, n_act=act.size)
    h = 1e-6
    noise = 1e-14 * (abs(loss(st)) + 1.0) / h  # rounding floor of a central difference

    def close(fd, ad, ref):
        return abs(fd - ad) <= 1e-5 * (abs(fd) + 1e-2 * ref) + noise

    for k in range(4):
        arr = st.arrays()[k]
        for _ in range(6):
            idx = tuple(rng.integers(0, d) for d in arr.shape)
            sp_, sm_ = st.copy(), st.copy()
            sp_.arrays()[k][idx] += h
            sm_.arrays()[k][idx] -= h
            fd = (loss(sp_) - loss(sm_)) / (2 * h)
            assert close(fd, adj[k][idx], np.abs(adj[k]).max()), (name, k, idx, fd, adj[k][idx])
    for i in range(4):
        e = np.zeros(4)
        e[i] = h
        fdq = (loss(st, qq=q + e) - loss(st, qq=q - e)) / (2 * h)
        fdu = (loss(st, uu=u + e) - loss(st, uu=u - e)) / (2 * h)
        assert close(fdq, qb[i], np.abs(qb).max()), (name, "q", i, fdq, qb[i])
        assert close(fdu, ub[i], np.abs(ub).max()), (name, "u", i, fdu, ub[i])
    if sp.material == orc.MAT["muscle"]:
        for j in range(act.size):
            e = np.zeros(act.size)
            e[j] = h
            fda = (loss(st, aa=act + e) - loss(st, aa=act - e)) / (2 * h)
            assert close(fda, ab[j], np.abs(ab).max()), (name, "a", j)


def test_substep_adjoint_dot_product():
    """<J d, w> = <d, J^T w> with J d by a directional central difference."""
    sp, st, q, u, act = _tiny_case("box_ground", seed=3)
    rng = np.random.default_rng(5)
    wts = [rng.standard_normal(a.shape) for a in st.arrays()]
    dirs = [rng.standard_normal(a.shape) for a in st.arrays()]
    adj, _, _, _ = orc.substep_adj(sp, st, wts, q, u, act, n_act=act.size)
    h = 1e-7
    sp_, sm_ = st.copy(), st.copy()
    for k in range(4):
        sp_.arrays()[k][...] += h * dirs[k]
        sm_.arrays()[k][...] -= h * dirs[k]
    op, _ = orc.substep(sp, sp_, q, u, act)
    om, _ = orc.substep(sp, sm_, q, u, act)
    lhs = sum(((a - b) / (2 * h) * w).sum() for a, b, w in zip(op.arrays(), om.arrays(), wts))
    rhs = sum((a * d).sum() for a, d in zip(adj, dirs))
    assert abs(lhs - rhs) < 1e-6 * abs(rhs)


@pytest.mark.parametrize("name,reward", [("capsule", "flat"), ("container", "reach"), ("muscle", "jump")])
def test_rollout_adjoint_fd(name, reward):
    """Checkpointed reverse of a 2-control-step rollout (rewards on every step, loss on the
    final state): action, initial-state and initial-pose gradients vs central differences."""
    rng = np.random.default_rng(21)
    kw = dict(CASES[name])
    n_coll = 0 if kw.get("collider", "none") == "none" else 3
    if n_coll:
        kw.update(act_map=(0, 2, 3) if name == "capsule" else (0, 1, 2), act_scale=(0.01, 0.01, 0.05))
    kw.update(reward=reward, n_sub=6, rparam=(0.3, 3.0, 1e-2, 0) if reward != "reach" else (0.5, 0.45, 0.4, 0),
              substeps=3)
    sp = spec_for(G=8, dt=2e-3, bound=2, **kw)
    st = _rand_state(10, 8, rng, lo=0.3, hi=0.7, vs=0.5)
    if name == "container":
        st.F = np.broadcast_to(np.eye(3), st.F.shape).copy()
    st.group = rng.integers(-1, 4, 10).astype(np.int32)
    # off the node lattice: at q = (0.5, 0.5, .) nodes sit on the container's medial planes,
    # where the SDF normal jumps and central differences are meaningless
    q0 = np.array([0.5031, 0.4967, 0.4043, 0.1])
    A = n_coll + sp.n_groups
    acts = rng.uniform(-1, 1, (2, A))
    rbar = rng.standard_normal(2)
    xw = rng.standard_normal((10, 3))

    def loss(s, qq=q0, aa=acts):
        o, _, rw, _ = orc.rollout(sp, s, qq, aa)
        return (rw * rbar).sum() + (o.x * xw).sum()

    ag, (xb, vb, Cb, Fb), qb = orc.rollout_adj(sp, st, q0, acts, adj_final=(xw, None, None, None), rbar=rbar)
    h = 1e-6
    noise = 1e-14 * (abs(loss(st)) + 1.0) / h

    def close(fd, ad, ref):
        return abs(fd - ad) <= 1e-5 * (abs(fd) + 1e-2 * ref) + noise

    for t in range(2):
        for j in range(A):
            ap, am = acts.copy(), acts.copy()
            ap[t, j] += h
            am[t, j] -= h
            fd = (loss(st, aa=ap) - loss(st, aa=am)) / (2 * h)
            assert close(fd, ag[t, j], np.abs(ag).max()), (t, j, fd, ag[t, j])
    for k, g in enumerate((xb, vb, Cb, Fb)):
        for _ in range(4):
            idx = tuple(rng.integers(0, d) for d in g.shape)
            sp_, sm_ = st.copy(), st.copy()
            sp_.arrays()[k][idx] += h
            sm_.arrays()[k][idx] -= h
            fd = (loss(sp_) - loss(sm_)) / (2 * h)
            assert close(fd, g[idx], np.abs(g).max()), (k, idx, fd, g[idx])
    for i in range(4):
        e = np.zeros(4)
        e[i] = h
        fd = (loss(st, qq=q0 + e) - loss(st, qq=q0 - e)) / (2 * h)
        assert close(fd, qb[i], np.abs(qb).max()), (i, fd, qb[i])


# ------------------------------------------------------------------ rewards (App. E)

def test_reward_closed_forms():
    st = orc.State(np.array([[0.5, 0.5, 0.1], [0.4, 0.5, 0.1], [0.3, 0.2, 0.3]]), np.array([[1.0, 0, 0], [3.0, 0, 0],
                                                                                             [9.0, 0, 0]]),
                   np.zeros((3, 3, 3)), np.broadcast_to(np.eye(3), (3, 3, 3)))
    flat = spec_for(reward="flat", n_sub=2, rparam=(0.125, 0, 0, 0))
    d = 0.1 / 0.125
    assert abs(orc.reward(flat, st, np.zeros(4), np.zeros(1)) - (1 / (1 + d)) ** 2) < 1e-14
    reach = spec_for(reward="reach", rparam=(0.5, 0.5, 0.5, 0))
    q = np.array([0.6, 0.5, 0.5, 0.0])
    assert abs(orc.reward(reach, st, q, np.zeros(1)) - 2 * (1 / 1.01) ** 2) < 1e-14
    q = np.array([0.8, 0.5, 0.5, 0.0])
    assert abs(orc.reward(reach, st, q, np.zeros(1)) - (1 / 1.09) ** 2) < 1e-14
    jump = spec_for("muscle", reward="jump", n_sub=2, rparam=(0.05, 3.0, 1e-4, 0), n_groups=2)
    a = np.array([0.5, -1.0])
    assert abs(orc.reward(jump, st, np.zeros(4), a) - (2.0 + 3.0 * 0.05 - 1e-4 * 1.25)) < 1e-14


# ------------------------------------------------------------------ binning (bit-exact reference)

def test_binning_keys_and_stable_sort():
    """Cell base from FP32 x with separate roundings: base = floor(x*G - 0.5), so the
    particle lies in [ (base+0.5) dx, (base+1.5) dx ); key is tile-major with 4^3 tiles.
    The counting sort is a stable permutation (checked against numpy's stable argsort)."""
    G = 32
    x = (0.1 + 0.8 * RNG.random((5000, 3))).astype(np.float32)
    x[:50] = (np.floor(x[:50] * G - 0.5) + 0.5).astype(np.float32) / G  # exactly on cell boundaries
    keys = orc.bin_keys_f32(x, G)
    tile, cell = keys // 64, keys % 64
    TG = G // 4
    b = np.stack([(tile % TG) * 4 + cell % 4, ((tile // TG) % TG) * 4 + (cell // 4) % 4,
                  (tile // (TG * TG)) * 4 + cell // 16], -1)
    # the same cell base from numpy float32 arithmetic, one rounding per operation (numpy
    # never fuses a multiply and a subtract), compared with no slack
    Xf = np.multiply(x, np.float32(G), dtype=np.float32)
    exp = np.clip(np.floor(np.subtract(Xf, np.float32(0.5), dtype=np.float32)).astype(np.int64), 0, G - 3)
    assert np.array_equal(b, exp)
    # and the particle lies in its cell's half-open support interval [b + 0.5, b + 1.5) in the
    # FP32 coordinate the key was made from
    assert np.all(b + 0.5 <= Xf) and np.all(Xf < b + 1.5)
    perm = orc.stable_sort(keys)
    assert np.array_equal(np.sort(perm), np.arange(5000))
    assert np.array_equal(perm, np.argsort(keys, kind="stable"))


# ------------------------------------------------------------------ observations (App. E)

def test_observation_definition_invariants():
    """x' is the first n_sub particles, the mean is their centroid (translation moves both by
    the shift), the pose entries follow the action map, the target fills only REACH."""
    rng = np.random.default_rng(31)
    sp = spec_for(collider="capsule", coll_dims=(0.03, 0.1, 0, 0), act_map=(0, 2, 3),
                  act_scale=(0.01, 0.01, 0.05), reward="flat", n_sub=5, rparam=(0.2, 0, 0, 0))
    x = rng.random((9, 3))
    q = np.array([0.1, 0.2, 0.3, 0.4])
    o = orc.observe(sp, x, q)
    assert o.shape == (3 * 5 + 10,)
    assert np.array_equal(o[:15].reshape(5, 3), x[:5])
    shift = np.array([0.05, -0.02, 0.01])
    o2 = orc.observe(sp, x + shift, q)
    assert np.allclose(o2[15:18] - o[15:18], shift, atol=1e-15)
    assert np.allclose(o[15:18], x[:5].mean(0), atol=1e-15)
    assert np.array_equal(o[18:22], [0.1, 0.3, 0.4, 0.0])
    assert np.array_equal(o[22:], [0.0, 0.0, 0.0])
    reach = spec_for(collider="box", coll_dims=(0.05, 0.05, 0.05, 0), act_map=(0, 1, 2),
                     act_scale=(0.01, 0.01, 0.01), reward="reach", n_sub=20, rparam=(0.5, 0.45, 0.4, 0))
    o3 = orc.observe(reach, x, q)  # fewer particles than n_sub: all of them
    assert o3.shape == (3 * 9 + 10,)
    assert np.array_equal(o3[-3:], [0.5, 0.45, 0.4])


@pytest.mark.parametrize("name", ["capsule", "container"])
def test_observation_adjoint_fd(name):
    """Adjoints of the observations at every control-step boundary injected into the
    checkpointed reverse pass: gradients of L = sum_t <c_t, obs(s_t)> with respect to the
    actions, the initial state and the initial pose against central differences."""
    rng = np.random.default_rng(33)
    kw = dict(CASES[name])
    kw.update(act_map=(0, 2, 3) if name == "capsule" else (0, 1, 2), act_scale=(0.01, 0.01, 0.05),
              reward="flat" if name == "capsule" else "reach", n_sub=6,
              rparam=(0.3, 0, 0, 0) if name == "capsule" else (0.5, 0.45, 0.4, 0), substeps=3)
    sp = spec_for(G=8, dt=2e-3, bound=2, **kw)
    st = _rand_state(10, 8, rng, lo=0.3, hi=0.7, vs=0.5)
    if name == "container":
        st.F = np.broadcast_to(np.eye(3), st.F.shape).copy()
    st.group = rng.integers(-1, 4, 10).astype(np.int32)
    q0 = np.array([0.5031, 0.4967, 0.4043, 0.1])
    T = 2
    A = 3 + sp.n_groups
    acts = rng.uniform(-1, 1, (T, A))
    od = orc.obs_dim(sp, 10)
    cw = rng.standard_normal((T + 1, od))

    def loss(s, qq=q0, aa=acts):
        cur, q = s.copy(), np.array(qq, np.float64)
        total = (cw[0] * orc.observe(sp, cur.x, q)).sum()
        for t in range(T):
            cur, q, _, _ = orc.rollout(sp, cur, q, aa[t:t + 1])
            total += (cw[t + 1] * orc.observe(sp, cur.x, q)).sum()
        return total

    ag, (xb, vb, Cb, Fb), qb = orc.rollout_adj(sp, st, q0, acts, obs_adj=cw)
    h = 1e-6
    noise = 1e-14 * (abs(loss(st)) + 1.0) / h

    def close(fd, ad, ref):
        return abs(fd - ad) <= 1e-5 * (abs(fd) + 1e-2 * ref) + noise

    for t in range(T):
        for j in range(A):
            ap, am = acts.copy(), acts.copy()
            ap[t, j] += h
            am[t, j] -= h
            fd = (loss(st, aa=ap) - loss(st, aa=am)) / (2 * h)
            assert close(fd, ag[t, j], np.abs(ag).max()), (t, j, fd, ag[t, j])
    for k, g in enumerate((xb, vb, Cb, Fb)):
        for _ in range(4):
            idx = tuple(rng.integers(0, d) for d in g.shape)
            sp_, sm_ = st.copy(), st.copy()
            sp_.arrays()[k][idx] += h
            sm_.arrays()[k][idx] -= h
            fd = (loss(sp_) - loss(sm_)) / (2 * h)
            assert close(fd, g[idx], np.abs(g).max()), (k, idx, fd, g[idx])
    for i in range(4):
        e = np.zeros(4)
        e[i] = h
        fd = (loss(st, qq=q0 + e) - loss(st, qq=q0 - e)) / (2 * h)
        assert close(fd, qb[i], np.abs(qb).max()), (i, fd, qb[i])


# ------------------------------------------------------------------ multi-capsule collider

def _caps_spec(n_caps=3, **kw):
    base = dict(G=8, dt=2e-3, bound=2, collider="capsules", n_caps=n_caps, coll_dims=(0.06, 0.1, 0, 0),
                cap_offset=(0.0, 0.13, 0.0), act_scale=(0.01, 0.01, 0.01, 0.05), coll_mu=0.4, substeps=3,
                pose0=(0.5031, 0.3667, 0.4043, 0.1))
    base.update(kw)
    return base


def test_capsule_union_is_nearest_capsule():
    """The union of capsules answers like the nearest single capsule (distance, normal,
    Hessian, body velocity), and one capsule is the single-capsule collider."""
    rng = np.random.default_rng(51)
    es = wl.EnvSpec(n_particles=1, grid_res=8, substeps=1, dt=1e-4, **{k: v for k, v in _caps_spec().items()
                                                                        if k not in ("G", "dt", "substeps")})
    sp = orc.make_spec(es)
    one = spec_for(collider="capsule", coll_dims=(0.06, 0.1, 0, 0))
    q = orc.initial_pose(es) + 0.01 * rng.standard_normal(12)
    u = rng.standard_normal(12)
    for _ in range(40):
        xw = 0.3 + 0.4 * rng.random(3)
        d, n, H, vb = orc.collider(sp, xw, q, u)
        singles = [orc.collider(one, xw, q[4 * j:4 * j + 4], u[4 * j:4 * j + 4]) for j in range(3)]
        j = int(np.argmin([t[0] for t in singles]))
        assert d == singles[j][0]
        assert np.array_equal(n, singles[j][1]) and np.array_equal(H, singles[j][2])
        assert np.array_equal(vb, singles[j][3])
    # n_caps = 1 rollout equals the single-capsule rollout
    kw = _caps_spec(n_caps=1)
    es1 = wl.EnvSpec(n_particles=10, grid_res=8, substeps=3, dt=2e-3, **{k: v for k, v in kw.items()
                                                                         if k not in ("G", "dt", "substeps")})
    esc = es1.replace(collider="capsule", n_caps=0, act_map=(0, 1, 2, 3))
    st = _rand_state(10, 8, rng, lo=0.3, hi=0.7, vs=0.5)
    acts = rng.uniform(-1, 1, (2, 4))
    a1, q1, r1, _ = orc.rollout(orc.make_spec(es1), st, orc.initial_pose(es1), acts)
    a2, q2, r2, _ = orc.rollout(orc.make_spec(esc), st, np.array(esc.pose0, np.float64), acts)
    assert np.array_equal(a1.x, a2.x) and np.array_equal(q1, q2)


def test_capsules_rollout_adjoint_fd():
    """Checkpointed reverse with three independently driven capsules (12 collider actions per
    step, a 12-entry pose): action, initial-state and initial-pose gradients against central
    differences."""
    rng = np.random.default_rng(53)
    kw = _caps_spec()
    es = wl.EnvSpec(n_particles=10, grid_res=8, substeps=3, dt=2e-3, material="neohookean", E=1e4, nu=0.3,
                    rho=1e3, p_vol=1e-6, reward="flat", n_sub=6, rparam=(0.3, 0, 0, 0),
                    **{k: v for k, v in kw.items() if k not in ("G", "dt", "substeps")})
    sp = orc.make_spec(es)
    st = _rand_state(10, 8, rng, lo=0.3, hi=0.7, vs=0.5)
    q0 = orc.initial_pose(es)
    T, A = 2, 12
    acts = rng.uniform(-1, 1, (T, A))
    rbar = rng.standard_normal(T)
    xw = rng.standard_normal((10, 3))

    def loss(s, qq=q0, aa=acts):
        o, _, rw, _ = orc.rollout(sp, s, qq, aa)
        return (rw * rbar).sum() + (o.x * xw).sum()

    ag, (xb, vb, Cb, Fb), qb = orc.rollout_adj(sp, st, q0, acts, adj_final=(xw, None, None, None), rbar=rbar)
    assert qb.shape == (12,) and np.abs(ag).max() > 0
    h = 1e-6
    noise = 1e-14 * (abs(loss(st)) + 1.0) / h

    def close(fd, ad, ref):
        return abs(fd - ad) <= 1e-5 * (abs(fd) + 1e-2 * ref) + noise

    for t in range(T):
        for j in range(A):
            ap, am = acts.copy(), acts.copy()
            ap[t, j] += h
            am[t, j] -= h
            fd = (loss(st, aa=ap) - loss(st, aa=am)) / (2 * h)
            assert close(fd, ag[t, j], np.abs(ag).max()), (t, j, fd, ag[t, j])
    for k, g in enumerate((xb, vb, Cb, Fb)):
        for _ in range(3):
            idx = tuple(rng.integers(0, d) for d in g.shape)
            sp_, sm_ = st.copy(), st.copy()
            sp_.arrays()[k][idx] += h
            sm_.arrays()[k][idx] -= h
            fd = (loss(sp_) - loss(sm_)) / (2 * h)
            assert close(fd, g[idx], np.abs(g).max()), (k, idx, fd, g[idx])
    for i in range(12):
        e = np.zeros(12)
        e[i] = h
        fd = (loss(st, qq=q0 + e) - loss(st, qq=q0 - e)) / (2 * h)
        assert close(fd, qb[i], np.abs(qb).max()), (i, fd, qb[i])
    # every capsule takes part in the contact
    assert all(np.abs(qb[4 * j:4 * j + 3]).max() > 0 for j in range(3))


# ------------------------------------------------------------------ symmetries of a substep (App. D.3)

_RZ = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])  # quarter turn about z


def _rotate(st, c):
    """The state turned a quarter about the vertical axis through (c/2, c/2): points
    (x, y, z) -> (c - y, x, z), vectors by _RZ, matrices by _RZ M _RZ^T."""
    x = np.stack([c - st.x[:, 1], st.x[:, 0], st.x[:, 2]], 1)
    out = orc.State(x, st.v @ _RZ.T, _RZ @ st.C @ _RZ.T, _RZ @ st.F @ _RZ.T, st.group)
    return out


def _rotate_pose(q, u, c):
    return (np.array([c - q[1], q[0], q[2], q[3] + np.pi / 2]), np.array([-u[1], u[0], u[2], u[3]]))


@pytest.mark.parametrize("name", list(CASES))
def test_substep_quarter_turn_equivariance(name):
    """A substep commutes with a quarter turn about the vertical axis through the centre of
    the node lattice, which maps nodes onto nodes (i, j) -> (G-1-j, i) and the quadratic
    B-spline stencil onto itself: the materials are isotropic (the muscle fibre is vertical),
    gravity and the ground are vertical, the walls are symmetric, and the collider turns with
    its pose.  Any mixed-up axis or index in P2G, the grid update or G2P breaks this."""
    sp, st, q, u, act = _tiny_case(name, seed=23)
    c = (sp.G - 1) / sp.G
    out, s0 = orc.substep(sp, st, q, u, act)
    qr, ur = _rotate_pose(q, u, c)
    out_r, s1 = orc.substep(sp, _rotate(st, c), qr, ur, act)
    assert s0 == 0 and s1 == 0
    want = _rotate(out, c)
    for k, (a, b) in enumerate(zip(out_r.arrays(), want.arrays())):
        assert np.abs(a - b).max() <= 1e-11 * max(np.abs(b).max(), 1.0), (name, k, np.abs(a - b).max())
    # the substep moved something (the comparison is not between two unchanged states)
    assert np.abs(out.v - st.v).max() > 1e-6


@pytest.mark.parametrize("name", list(CASES))
def test_substep_whole_cell_translation_invariance(name):
    """Away from the walls, shifting the particles and the collider by whole cells shifts
    the result by the same amount and leaves v, C and F unchanged (weights depend only on
    positions relative to the node lattice)."""
    kw = dict(CASES[name])
    rng = np.random.default_rng(29)
    G = 32
    sp = spec_for(G=G, dt=2e-3, bound=2, **kw)
    st = _rand_state(12, G, rng, lo=0.4, hi=0.6, vs=0.5)
    if name == "container":
        st.F = np.broadcast_to(np.eye(3), st.F.shape) * np.cbrt(1 + 0.02 * rng.standard_normal((12, 1, 1)))
    st.group = rng.integers(-1, 4, 12).astype(np.int32)
    q = np.array([0.5, 0.5, 0.42, 0.2]) + 0.02 * rng.standard_normal(4)
    u = 0.3 * rng.standard_normal(4)
    act = np.concatenate([np.zeros(len(kw.get("act_map", ()))), rng.uniform(-1, 1, 4)])
    shift = np.array([3.0, -2.0, 1.0]) / G
    out, s0 = orc.substep(sp, st, q, u, act)
    moved = st.copy()
    moved.x = st.x + shift
    out_m, s1 = orc.substep(sp, moved, q + np.append(shift, 0.0), u, act)
    assert s0 == 0 and s1 == 0
    assert np.abs(out_m.x - (out.x + shift)).max() < 1e-13
    for a, b in ((out_m.v, out.v), (out_m.C, out.C), (out_m.F, out.F)):
        assert np.abs(a - b).max() <= 1e-10 * max(np.abs(b).max(), 1.0)
    assert np.abs(out.v - st.v).max() > 1e-6


@pytest.mark.parametrize("material", ["neohookean", "vonmises", "muscle", "fluid"])
def test_substep_preserves_affine_velocity(material):
    """APIC through a whole substep (P2G, grid update, G2P): particles at rest shape (F = I, so
    no stress) carrying an affine field v_p = a + B x_p with C_p = B keep it exactly, with no
    gravity and away from the walls: P2G gives m_i (a + B x_i) on every node and G2P reads
    it back.  For the fluid B is a rotation rate, since its viscosity acts on C + C^T."""
    rng = np.random.default_rng(37)
    G = 16
    sp = spec_for(material, G=G, dt=1e-3, bound=3, gravity=(0.0, 0.0, 0.0))
    n = 40
    x = 0.35 + 0.3 * rng.random((n, 3))
    a = rng.standard_normal(3)
    B = rng.standard_normal((3, 3))
    if material == "fluid":
        B = B - B.T
    st = orc.State(x, a + x @ B.T, np.broadcast_to(B, (n, 3, 3)), np.broadcast_to(np.eye(3), (n, 3, 3)))
    out, status = orc.substep(sp, st, act=np.zeros(4))
    assert status == 0
    assert np.abs(out.v - (a + st.x @ B.T)).max() <= 1e-12 * np.abs(st.v).max()
    assert np.abs(out.C - B).max() <= 1e-10 * np.abs(B).max()
    assert np.abs(out.x - (st.x + sp.dt * out.v)).max() <= 1e-15


@pytest.mark.parametrize("collider,act_map", [("capsule", (0, 2, 3)), ("box", (0, 1, 2)), ("capsules", ())])
def test_collider_pose_follows_relative_actions(collider, act_map):
    """Actions are relative poses per control step (App. E): over a control step's S
    substeps the pose moves at the constant rate s_a a / (S dt), so after each step it has
    moved by exactly s_a a (summed into the mapped components; capsule j of a union by its
    own four actions)."""
    rng = np.random.default_rng(41)
    kw = dict(collider=collider, coll_dims=(0.03, 0.1, 0.05, 0), act_scale=(0.01, 0.02, 0.03, 0.05),
              pose0=(0.5, 0.5, 0.8, 0.1))
    if collider == "capsules":
        kw.update(n_caps=3, cap_offset=(0.0, 0.1, 0.0))
    else:
        kw.update(act_map=act_map)
    es = wl.EnvSpec(n_particles=8, grid_res=16, substeps=7, dt=1e-4, material="neohookean", E=1e4, nu=0.3, rho=1e3,
                    p_vol=1e-6, **kw)
    sp = orc.make_spec(es)
    st = _rand_state(8, 16, rng, lo=0.3, hi=0.4)  # far below the bodies: no contact
    T, A = 3, es.action_dim
    acts = rng.uniform(-1.0, 1.0, (T, A))
    q0 = orc.initial_pose(es)
    _, q, _, status = orc.rollout(sp, st, q0, acts)
    assert status == 0
    want = q0.copy()
    for t in range(T):
        for j in range(A):
            comp = j if collider == "capsules" else act_map[j]
            want[comp] += es.act_scale[j % 4] * acts[t, j]
    assert np.abs(q - want).max() <= 1e-14
