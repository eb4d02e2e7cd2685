"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
published known-answer vectors, closed forms, identities, brute force.

Each test names the fact it uses. A plausible slip in the oracle (a dropped term,
a wrong sign, a transposed operand) breaks at least one of them:
  FK              closed-form chain poses
  M (CRBA)        analytic planar-chain inertia; KE identity from finite-differenced
                  FK; M e_i = ID(q, 0, e_i) columns (spec requirement)
  bias (RNE)      Lagrangian form by finite differences of M and of the potential
  LTDL            reconstruction, no fill outside the ancestor pattern, numpy solve
  dynamics        pendulum periods (small angle, discrete-time closed form), three-link
                  linearised modes, free fall, momentum, symmetric spin
  collision       surface sampling of spheres / capsules / boxes against a plane
  constraint      brute-force active-set enumeration (frictionless), Moreau /
  solve           complementarity conditions of the elliptic cone (friction),
                  resting-contact penetration fixed point and force balance,
                  Coulomb sliding deceleration
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import Oracle
from paper_2601_22074_b300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    out = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *v = line.split()
            out[k] = [float(x) for x in v]
    return out


# ----------------------------------------------------------------------------- helpers
def quat_mul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def advance_qpos(spec, q, v, dt):
    """Move qpos along qvel for time dt (free joints: world translation, body-frame
    rotation by the exponential map), the meaning of qvel in the model convention."""
    q = np.array(q, dtype=float)
    qa, da = spec.jnt_qposadr(), spec.jnt_dofadr()
    for j, t in enumerate(spec.jnt_type):
        a, d = qa[j], da[j]
        if t == I.FREE:
            q[a:a + 3] += dt * v[d:d + 3]
            w = np.asarray(v[d + 3:d + 6]) * dt
            ang = np.linalg.norm(w)
            if ang > 0:
                dq = np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * w / ang])
                q[a + 3:a + 7] = quat_mul(q[a + 3:a + 7], dq)
        else:
            q[a] += dt * v[d]
    return q


def armature(spec):
    arm = np.zeros(spec.nv)
    da = spec.jnt_dofadr()
    for j, t in enumerate(spec.jnt_type):
        if t != I.FREE:
            arm[da[j]] = spec.jnt_armature[j]
    return arm


def ancestor_pattern(spec):
    """P[i, j] = True when dof j is dof i or one of its ancestors along the body tree."""
    body_of_dof = []
    for j, t in enumerate(spec.jnt_type):
        body_of_dof += [spec.jnt_body[j]] * (6 if t == I.FREE else 1)
    nv = len(body_of_dof)
    P = np.zeros((nv, nv), dtype=bool)
    for i in range(nv):
        for j in range(i + 1):
            b = body_of_dof[i]
            while b > 0 and b != body_of_dof[j]:
                b = spec.body_parent[b]
            P[i, j] = b == body_of_dof[j] and b > 0
    return P


def random_state(spec, rng, qscale=0.5, vscale=1.0):
    q = spec.qpos_reset.copy()
    qa = spec.jnt_qposadr()
    for j, t in enumerate(spec.jnt_type):
        if t == I.FREE:
            q[qa[j]:qa[j] + 3] += rng.normal(0, 0.2, 3)
            qq = rng.normal(size=4)
            q[qa[j] + 3:qa[j] + 7] = qq / np.linalg.norm(qq)
        else:
            q[qa[j]] += rng.uniform(-qscale, qscale)
    v = rng.normal(0, vscale, spec.nv)
    return q, v


SPECS = {
    "pendulum": lambda: I.pendulum(3),
    "spatial_chain": I.spatial_chain,
    "quadruped": I.quadruped,
    "humanoid": I.humanoid,
    "manipulation_arm": None,  # filled below once box-box lands
}


# ----------------------------------------------------------------------------- Philox
def test_philox_known_answers():
    path = os.path.join(GOLD, "philox4x32_10_kat.txt")
    n = 0
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            out = Oracle.philox(w[0:4], w[4:6])
            assert out.tolist() == w[6:10]
            n += 1
    assert n == 3


# ----------------------------------------------------------------------------- FK
def chain_closed_form(q, L=0.3):
    """Planar chain about +y, links along -z at q=0: origins and COMs in closed form."""
    phi = np.cumsum(q)
    origins, coms = [], []
    o = np.zeros(3)
    for i in range(len(q)):
        u = np.array([-math.sin(phi[i]), 0.0, -math.cos(phi[i])])
        origins.append(o.copy())
        coms.append(o + 0.5 * L * u)
        o = o + L * u
    return np.array(origins), np.array(coms)


def test_fk_planar_chain_closed_form():
    spec = I.pendulum(3)
    o = Oracle(spec)
    rng = np.random.default_rng(1)
    for _ in range(5):
        q = rng.uniform(-math.pi, math.pi, 3)
        k = o.fk(q)
        origins, coms = chain_closed_form(q)
        np.testing.assert_allclose(k["xpos"][1:], origins, atol=1e-14)
        np.testing.assert_allclose(k["xipos"][1:], coms, atol=1e-14)
        # orientation: rotation about y by the absolute angle
        phi = np.cumsum(q)
        for i in range(3):
            R = k["xmat"][i + 1]
            c, s = math.cos(phi[i]), math.sin(phi[i])
            np.testing.assert_allclose(R, [[c, 0, s], [0, 1, 0], [-s, 0, c]], atol=1e-14)


# ----------------------------------------------------------------------------- mass matrix
def planar_chain_M(q, m=1.0, L=0.3, r=0.02):
    n = len(q)
    It = m * (3 * r * r + L * L) / 12
    phi = np.cumsum(q)
    c = np.array([[L if j < i else (L / 2 if j == i else 0.0) for j in range(n)]
                  for i in range(n)])
    Mabs = np.zeros((n, n))
    for j in range(n):
        for k in range(n):
            Mabs[j, k] = m * np.sum(c[:, j] * c[:, k]) * math.cos(phi[j] - phi[k])
    Mabs += It * np.eye(n)
    T = np.tril(np.ones((n, n)))
    return T.T @ Mabs @ T


def test_mass_matrix_planar_chain_analytic():
    spec = I.pendulum(3)
    o = Oracle(spec)
    rng = np.random.default_rng(2)
    for _ in range(5):
        q = rng.uniform(-math.pi, math.pi, 3)
        np.testing.assert_allclose(o.mass_matrix(q), planar_chain_M(q), atol=1e-14, rtol=1e-12)


@pytest.mark.parametrize("name", ["spatial_chain", "quadruped", "humanoid"])
def test_mass_matrix_spd_and_inverse_dynamics_columns(name):
    spec = SPECS[name]()
    o = Oracle(spec)
    rng = np.random.default_rng(3)
    for trial in range(3):
        q, v = random_state(spec, rng)
        ms = rng.uniform(0.8, 1.2, spec.nbody) if trial == 2 else None
        M = o.mass_matrix(q, ms)
        np.testing.assert_allclose(M, M.T, atol=1e-13)
        assert np.linalg.eigvalsh(M).min() > 0
        zero = np.zeros(spec.nv)
        base = o.rne(q, zero, zero, gravity=False, mass_scale=ms)
        np.testing.assert_allclose(base, 0.0, atol=1e-14)
        for i in range(spec.nv):
            e = np.zeros(spec.nv)
            e[i] = 1.0
            # rigid-body inverse dynamics: armature (rotor inertia) is added on the diagonal
            col = o.rne(q, zero, e, gravity=False, mass_scale=ms) + armature(spec) * e
            np.testing.assert_allclose(col, M[:, i], atol=1e-12 * np.abs(M).max())


@pytest.mark.parametrize("name", ["spatial_chain", "humanoid"])
def test_kinetic_energy_from_fk_finite_differences(name):
    """1/2 qdot^T M qdot equals sum_b 1/2 m |c_dot|^2 + 1/2 w^T I_w w, with c_dot and w
    obtained by finite differences of the FK poses along the motion."""
    spec = SPECS[name]()
    o = Oracle(spec)
    rng = np.random.default_rng(4)
    q, v = random_state(spec, rng)
    eps = 1e-6
    kp_, km_ = o.fk(advance_qpos(spec, q, v, eps)), o.fk(advance_qpos(spec, q, v, -eps))
    k0 = o.fk(q)
    ke = 0.0
    for b in range(1, spec.nbody):
        m = spec.body_mass[b]
        cd = (kp_["xipos"][b] - km_["xipos"][b]) / (2 * eps)
        Rd = (kp_["xmat"][b] - km_["xmat"][b]) / (2 * eps)
        W = Rd @ k0["xmat"][b].T
        w = np.array([W[2, 1], W[0, 2], W[1, 0]])
        Ib = spec.body_inertia[b]
        Ibm = np.array([[Ib[0], Ib[3], Ib[4]], [Ib[3], Ib[1], Ib[5]], [Ib[4], Ib[5], Ib[2]]])
        Iw = k0["xmat"][b] @ Ibm @ k0["xmat"][b].T
        ke += 0.5 * m * cd @ cd + 0.5 * w @ Iw @ w
    M = o.mass_matrix(q)
    ke_M = 0.5 * v @ (M - np.diag(armature(spec))) @ v
    assert abs(ke - ke_M) <= 1e-7 * abs(ke_M)


# ----------------------------------------------------------------------------- bias forces
@pytest.mark.parametrize("name", ["pendulum", "spatial_chain"])
def test_bias_equals_lagrangian_form(name):
    """bias = Mdot qdot - 1/2 d(qdot^T M qdot)/dq + dV/dq, V = -sum_b m_b g . c_b, all
    by central differences (fixed-base hinge/slide chains)."""
    spec = SPECS[name]()
    o = Oracle(spec)
    rng = np.random.default_rng(5)
    g = np.array(spec.opt.gravity)
    nv = spec.nv

    def V(q):
        k = o.fk(q)
        return -sum(spec.body_mass[b] * g @ k["xipos"][b] for b in range(1, spec.nbody))

    for _ in range(3):
        q, v = random_state(spec, rng)
        eps = 1e-5
        Mdot = (o.mass_matrix(q + eps * v) - o.mass_matrix(q - eps * v)) / (2 * eps)
        dT = np.zeros(nv)
        dV = np.zeros(nv)
        for k in range(nv):
            e = np.zeros(nv)
            e[k] = eps
            dT[k] = 0.5 * (v @ o.mass_matrix(q + e) @ v - v @ o.mass_matrix(q - e) @ v) / (2 * eps)
            dV[k] = (V(q + e) - V(q - e)) / (2 * eps)
        lag = Mdot @ v - dT + dV
        bias = o.rne(q, v, np.zeros(nv), gravity=True)
        np.testing.assert_allclose(bias, lag, atol=1e-7 * max(1.0, np.abs(lag).max()))


# ----------------------------------------------------------------------------- LTDL
@pytest.mark.parametrize("name", ["spatial_chain", "quadruped", "humanoid"])
def test_ltdl_reconstruction_pattern_and_solve(name):
    spec = SPECS[name]()
    o = Oracle(spec)
    rng = np.random.default_rng(6)
    q, _ = random_state(spec, rng)
    M = o.mass_matrix(q)
    L, D, rc = o.ltdl(M)
    assert rc == 0 and (D > 0).all()
    np.testing.assert_allclose(L.T @ np.diag(D) @ L, M, atol=1e-12 * np.abs(M).max())
    # no fill: L is nonzero only on (dof, ancestor dof) pairs of the kinematic tree
    struct = ancestor_pattern(spec)
    assert not np.any((np.abs(np.tril(L, -1)) > 0) & ~struct)
    assert not np.any((np.abs(M) > 0) & ~(struct | struct.T))
    nnz = int(np.count_nonzero(np.tril(struct)))
    if name == "humanoid":
        assert nnz == 341  # stored entries of the tree-sparse humanoid mass matrix
    b = rng.normal(size=spec.nv)
    np.testing.assert_allclose(o.ltdl_solve(L, D, b), np.linalg.solve(M, b), rtol=1e-9, atol=1e-12)


# ----------------------------------------------------------------------------- dynamics
def simulate(o, spec, q, v, nsteps, ctrl=None, **kw):
    qacc = np.zeros(spec.nv)
    traj = [(q.copy(), v.copy())]
    for _ in range(nsteps):
        r = o.step(q, v, qacc, ctrl, nsub=1, **kw)
        q, v, qacc = r["qpos"], r["qvel"], r["qacc"]
        traj.append((q.copy(), v.copy()))
    return traj, r


def crossing_period(x, h):
    """Mean period from upward zero crossings with linear interpolation."""
    t = []
    for i in range(len(x) - 1):
        if x[i] < 0 <= x[i + 1]:
            t.append((i + (-x[i]) / (x[i + 1] - x[i])) * h)
    d = np.diff(t)
    return float(np.mean(d))


def test_one_link_pendulum_small_angle_period():
    gold = golden("closed_forms.txt")
    spec = I.pendulum(1)
    o = Oracle(spec)
    h = spec.opt.timestep
    m, L, r, g = 1.0, 0.3, 0.02, 9.81
    Ip = m * (3 * r * r + L * L) / 12 + m * (L / 2) ** 2
    w = math.sqrt(m * g * (L / 2) / Ip)
    T_cont = 2 * math.pi / w
    assert abs(T_cont - gold["one_link_period_s"][0]) < 1e-5
    T_disc = 2 * math.pi * h / math.acos(1 - w * w * h * h / 2)
    traj, _ = simulate(o, spec, np.array([1e-4]), np.array([0.0]), 3000)
    x = np.array([s[0][0] for s in traj])
    T = crossing_period(x, h)
    assert abs(T - T_disc) < 2e-6 * T_disc
    assert abs(T - T_cont) < 1e-4 * T_cont


def test_three_link_linearised_modes():
    gold = golden("closed_forms.txt")
    spec = I.pendulum(3)
    o = Oracle(spec)
    n, m, L, r, g = 3, 1.0, 0.3, 0.02, 9.81
    c = np.array([[L if j < i else (L / 2 if j == i else 0.0) for j in range(n)] for i in range(n)])
    T = np.tril(np.ones((n, n)))
    K = T.T @ np.diag(m * g * c.sum(0)) @ T
    M0 = o.mass_matrix(np.zeros(3))
    np.testing.assert_allclose(M0, planar_chain_M(np.zeros(3)), atol=1e-14)
    # gravity stiffness from the oracle's bias by central differences
    eps = 1e-6
    Kq = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = eps
        Kq[:, k] = (o.rne(e, np.zeros(n), np.zeros(n)) - o.rne(-e, np.zeros(n), np.zeros(n))) / (2 * eps)
    np.testing.assert_allclose(Kq, K, rtol=1e-7, atol=1e-9)
    w2, modes = sl.eigh(K, M0)
    w = np.sqrt(w2)
    np.testing.assert_allclose(w, gold["three_link_omega_rad_s"], rtol=2e-6)
    np.testing.assert_allclose(2 * math.pi / w, gold["three_link_period_s"], rtol=2e-5)
    # simulate the first mode at small amplitude: its period follows the discrete closed form
    h = spec.opt.timestep
    v1 = modes[:, 0] / np.abs(modes[:, 0]).max() * 1e-4
    traj, _ = simulate(o, spec, v1.copy(), np.zeros(3), 4000)
    x = np.array([s[0] @ (M0 @ modes[:, 0]) for s in traj])
    Tm = crossing_period(x, h)
    Td = 2 * math.pi * h / math.acos(1 - w2[0] * h * h / 2)
    assert abs(Tm - Td) < 2e-5 * Td


def test_free_fall_closed_form():
    gold = golden("closed_forms.txt")
    spec = I.free_body(I.SPHERE, (0.1,), plane=False, timestep=0.005)
    o = Oracle(spec)
    q0 = spec.qpos_reset.copy()
    traj, _ = simulate(o, spec, q0, np.zeros(6), 100)
    q, v = traj[-1]
    np.testing.assert_allclose(q0[2] - q[2], gold["free_fall_n100_h5ms_drop_m"][0], atol=1e-12)
    np.testing.assert_allclose(-v[2], gold["free_fall_n100_h5ms_speed_m_s"][0], atol=1e-12)
    np.testing.assert_allclose(q[:2], q0[:2], atol=0)


def test_zero_gravity_free_body_momentum_and_symmetric_spin():
    # linear momentum is constant for a tumbling asymmetric body
    spec = I.free_body(I.BOX, (0.1, 0.2, 0.3), mass=2.0, plane=False, gravity=(0, 0, 0))
    o = Oracle(spec)
    v0 = np.array([0.3, -0.2, 0.1, 2.0, -1.0, 3.0])
    traj, _ = simulate(o, spec, spec.qpos_reset.copy(), v0, 500)
    for q, v in traj[::50]:
        np.testing.assert_allclose(v[:3], v0[:3], atol=1e-14)
    # a symmetric body spinning about its symmetry axis keeps its angular velocity
    spec2 = I.free_body(I.CAPSULE, (0.05, 0.2), plane=False, gravity=(0, 0, 0))
    o2 = Oracle(spec2)
    w0 = np.array([0, 0, 0, 0, 0, 7.0])
    traj2, _ = simulate(o2, spec2, spec2.qpos_reset.copy(), w0, 500)
    np.testing.assert_allclose(traj2[-1][1], w0, atol=1e-12)


def test_zero_gravity_quadruped_linear_momentum_rate_vanishes():
    """Internal PD torques only: d/dt (M qdot)[0:3] = (Mdot qdot + M qacc)[0:3] = 0."""
    spec = I.quadruped(gravity=(0, 0, 0))
    o = Oracle(spec)
    rng = np.random.default_rng(7)
    q, v = random_state(spec, rng)
    q[2] = 5.0  # far above the plane: no contacts
    ctrl = spec.qpos_reset[spec.act_qposadr()] + rng.normal(0, 0.5, spec.nu)
    r = o.step(q, v, np.zeros(spec.nv), ctrl, nsub=1)
    assert r["ncon"] == 0
    qacc = r["qacc"]
    eps = 1e-6
    Mdot = (o.mass_matrix(advance_qpos(spec, q, v, eps)) -
            o.mass_matrix(advance_qpos(spec, q, v, -eps))) / (2 * eps)
    M = o.mass_matrix(q)
    pdot = (Mdot @ v + M @ qacc)[:3]
    assert np.abs(pdot).max() < 1e-6 * np.abs(M @ qacc).max()


def test_pendulum_energy_drift_is_first_order_in_h():
    """Semi-implicit Euler on a chain with configuration-dependent M is not symplectic:
    mechanical energy drifts, but the drift over a fixed time is O(h) (a wrong bias or
    inertia term would leave an h-independent drift)."""
    drift = {}
    for h in (0.002, 0.0005):
        spec = I.pendulum(3, timestep=h)
        o = Oracle(spec)
        q = np.random.default_rng(8).uniform(-1, 1, 3)
        g = np.array(spec.opt.gravity)

        def energy(q, v):
            k = o.fk(q)
            return 0.5 * v @ o.mass_matrix(q) @ v - sum(
                spec.body_mass[b] * g @ k["xipos"][b] for b in range(1, 4))

        e0 = energy(q, np.zeros(3))
        traj, _ = simulate(o, spec, q, np.zeros(3), int(round(1.0 / h)))
        drift[h] = energy(*traj[-1]) - e0
    ratio = drift[0.002] / drift[0.0005]
    assert 3.3 < ratio < 4.7
    assert abs(drift[0.0005]) < 0.05


# ----------------------------------------------------------------------------- collision
def sample_surface(gtype, size, pos, R, n=40):
    pts = []
    if gtype == I.SPHERE:
        th, ph = np.meshgrid(np.linspace(0, math.pi, n), np.linspace(0, 2 * math.pi, n))
        loc = size[0] * np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1)
        pts = loc.reshape(-1, 3)
    elif gtype == I.CAPSULE:
        r, hl = size[0], size[1]
        th, ph = np.meshgrid(np.linspace(0, math.pi, n), np.linspace(0, 2 * math.pi, n))
        sph = r * np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1).reshape(-1, 3)
        pts = np.concatenate([sph + [0, 0, hl], sph - [0, 0, hl]])
    elif gtype == I.BOX:
        g = np.linspace(-1, 1, 9)
        a, b, c = np.meshgrid(g, g, g)
        cube = np.stack([a, b, c], -1).reshape(-1, 3)
        cube = cube[np.abs(cube).max(1) == 1]
        pts = cube * np.asarray(size)
    return pos + pts @ R.T


@pytest.mark.parametrize("gtype,size", [(I.SPHERE, (0.1,)), (I.CAPSULE, (0.05, 0.15)),
                                        (I.BOX, (0.1, 0.05, 0.2))])
def test_plane_contacts_against_surface_sampling(gtype, size):
    spec = I.free_body(gtype, size)
    o = Oracle(spec)
    rng = np.random.default_rng(9)
    for _ in range(20):
        q = spec.qpos_reset.copy()
        q[2] = rng.uniform(-0.05, 0.2)
        qq = rng.normal(size=4)
        q[3:7] = qq / np.linalg.norm(qq)
        k = o.fk(q)
        pts = sample_surface(gtype, size, k["gxpos"][1], k["gxmat"][1])
        zmin = pts[:, 2].min()
        con = o.collide(q)
        if zmin > 1e-9:
            assert len(con) == 0
            continue
        if len(con) == 0:
            assert zmin > -1e-9
            continue
        dist = con[:, 4]
        # the deepest contact equals the lowest surface point (sampling includes the
        # extreme points: sphere poles are hit only approximately)
        tol = 2e-3 * max(size) if gtype != I.BOX else 1e-12
        assert abs(dist.min() - zmin) <= tol
        for c in con:
            assert c[4] < 0
            np.testing.assert_allclose(c[8:11], [0, 0, 1], atol=0)   # plane normal
            np.testing.assert_allclose(c[7], 0.5 * c[4], atol=1e-12)  # midpoint depth
        if gtype == I.BOX:
            assert len(con) <= 4
            import itertools
            R, c = k["gxmat"][1], k["gxpos"][1]
            corners = np.array([c + R @ (np.array(sg) * size)
                                for sg in itertools.product((-1, 1), repeat=3)])
            below = np.sort(corners[:, 2][corners[:, 2] < 0])
            np.testing.assert_allclose(np.sort(dist), below[: len(dist)], atol=1e-12)


# ----------------------------------------------------------------------------- constraint solve
def random_problem(rng, nv, nc, mu):
    A = rng.normal(size=(nv, nv))
    M = A @ A.T + nv * np.eye(nv)
    a_s = rng.normal(size=nv) * 3
    J = rng.normal(size=(3 * nc, nv))
    aref = rng.normal(size=3 * nc)
    D = np.repeat(rng.uniform(0.5, 5.0, nc), 3)
    return M, a_s, J, aref, D, np.full(nc, mu)


def test_newton_frictionless_matches_active_set_enumeration():
    rng = np.random.default_rng(10)
    for trial in range(30):
        nv, nc = int(rng.integers(3, 7)), int(rng.integers(1, 5))
        M, a_s, J, aref, D, mu = random_problem(rng, nv, nc, 0.0)
        a, f, it = Oracle.newton(M, a_s, J, aref, D, mu)
        jn = J[0::3]
        an = aref[0::3]
        dn = D[0::3]
        best = None
        for mask in range(1 << nc):
            S = [c for c in range(nc) if mask >> c & 1]
            H = M.copy()
            rhs = M @ a_s
            for c in S:
                H += dn[c] * np.outer(jn[c], jn[c])
                rhs += dn[c] * an[c] * jn[c]
            x = np.linalg.solve(H, rhs)
            N = jn @ x - an
            if all(N[c] <= 1e-12 for c in S) and all(N[c] >= -1e-12 for c in range(nc) if c not in S):
                best = x
        assert best is not None
        np.testing.assert_allclose(a, best, rtol=1e-10, atol=1e-10)


def test_newton_friction_cone_optimality_conditions():
    rng = np.random.default_rng(11)
    for trial in range(30):
        nv, nc = int(rng.integers(3, 9)), int(rng.integers(1, 6))
        mu = float(rng.uniform(0.2, 1.5))
        M, a_s, J, aref, D, muv = random_problem(rng, nv, nc, mu)
        a, f, it = Oracle.newton(M, a_s, J, aref, D, muv)
        # stationarity: M (a - a_s) = J^T f
        np.testing.assert_allclose(M @ (a - a_s), J.T @ f, atol=1e-9 * max(1, np.abs(J.T @ f).max()))
        jar = J @ a - aref
        for c in range(nc):
            fc = f[3 * c:3 * c + 3]
            y = -jar[3 * c:3 * c + 3] - fc / D[3 * c]
            scale = max(1.0, np.abs(fc).max(), np.abs(y).max())
            # f in K_mu, y in the polar cone, f . y = 0 (Moreau decomposition of -jar)
            assert np.linalg.norm(fc[1:]) <= mu * fc[0] + 1e-9 * scale
            assert mu * np.linalg.norm(y[1:]) <= -y[0] + 1e-9 * scale
            assert abs(fc @ y) <= 1e-9 * scale * scale
        # the optimum has the lowest cost among perturbations
        c0 = Oracle.cost(M, a_s, J, aref, D, muv, a)
        for _ in range(5):
            assert Oracle.cost(M, a_s, J, aref, D, muv, a + 1e-4 * rng.normal(size=nv)) >= c0


def test_resting_sphere_penetration_and_force_balance():
    gold = golden("closed_forms.txt")
    for mass in (0.5, 4.0):
        spec = I.free_body(I.SPHERE, (0.1,), mass=mass, pos=(0, 0, 0.1))
        o = Oracle(spec)
        q, v = spec.qpos_reset.copy(), np.zeros(6)
        qacc = np.zeros(6)
        for _ in range(400):
            r = o.step(q, v, qacc, None, want_contacts=True)
            q, v, qacc = r["qpos"], r["qvel"], r["qacc"]
        con = r["contacts"]
        assert len(con) == 1
        assert abs(-con[0, 4] * 1e3 - gold["resting_penetration_mm"][0]) < 1e-5
        np.testing.assert_allclose(con[0, 18], mass * 9.81, rtol=1e-9)
        assert abs(con[0, 19]) < 1e-9 and abs(con[0, 20]) < 1e-9


def test_resting_box_force_balance():
    mass = 3.0
    spec = I.free_body(I.BOX, (0.1, 0.1, 0.05), mass=mass, pos=(0, 0, 0.05))
    o = Oracle(spec)
    q, v, qacc = spec.qpos_reset.copy(), np.zeros(6), np.zeros(6)
    for _ in range(400):
        r = o.step(q, v, qacc, None, want_contacts=True)
        q, v, qacc = r["qpos"], r["qvel"], r["qacc"]
    con = r["contacts"]
    assert len(con) == 4
    np.testing.assert_allclose(con[:, 18].sum(), mass * 9.81, rtol=1e-8)
    assert np.abs(con[:, 19:21]).max() < 1e-8 * mass * 9.81
    np.testing.assert_allclose(con[:, 18], mass * 9.81 / 4, rtol=1e-6)


def test_sliding_contacts_sit_on_the_cone_boundary():
    """Coulomb's law at sliding contacts: |f_t| = mu f_n with f_t opposing the slip.
    (With this soft elliptic model a kicked box partly lifts off because the cone
    projection of a large tangential reference acceleration raises f_n, so the
    deceleration is not mu g; the per-contact law is what the model fixes.)"""
    mu = 0.5
    spec = I.free_body(I.BOX, (0.1, 0.1, 0.05), mass=2.0, pos=(0, 0, 0.05), friction=mu)
    o = Oracle(spec)
    q, v, qacc = spec.qpos_reset.copy(), np.zeros(6), np.zeros(6)
    for _ in range(100):  # settle on the plane
        r = o.step(q, v, qacc, None)
        q, v, qacc = r["qpos"], r["qvel"], r["qacc"]
    v = v.copy()
    v[0] = 1.0
    nslide = 0
    for _ in range(200):
        k = o.fk(q)
        R, x = k["xmat"][1], k["xpos"][1]
        w = R @ v[3:6]
        r = o.step(q, v, qacc, None, want_contacts=True)
        for c in r["contacts"]:
            fn, ft = c[18], np.hypot(c[19], c[20])
            fw = c[21:24]
            vp = v[:3] + np.cross(w, c[5:8] - x)  # contact point velocity before the step
            vt = vp - vp[2] * np.array([0, 0, 1.0])
            if np.linalg.norm(vt) > 0.05 and fn > 0:
                nslide += 1
                np.testing.assert_allclose(ft, mu * fn, rtol=1e-9)
                assert fw[:2] @ vt[:2] < 0  # opposes the slip
        q, v, qacc = r["qpos"], r["qvel"], r["qacc"]
    assert nslide > 20
    assert abs(v[0]) < 1e-3 and q[0] > 0.05  # came to rest after sliding forward


# ----------------------------------------------------------------------------- reset
def test_reset_is_seeded_uniform_in_range():
    spec = I.pendulum(3)
    o = Oracle(spec)
    qs = np.array([o.reset(123, w)[0] for w in range(2000)])
    assert np.all(np.abs(qs) <= math.pi)
    np.testing.assert_allclose(qs.mean(0), 0, atol=0.15)
    np.testing.assert_allclose(qs.std(0), math.pi / math.sqrt(3), rtol=0.05)
    q1, _ = o.reset(123, 5)
    q2, _ = o.reset(123, 5)
    q3, _ = o.reset(124, 5)
    assert np.array_equal(q1, q2) and not np.array_equal(q1, q3)
    # the first hinge uses word 0 of counter {0, world, 1, 0}
    x = Oracle.philox([0, 5, 1, 0], [123, 0])
    np.testing.assert_allclose(q1[0], math.pi * (2 * (x[0] >> 8) / 2 ** 24 - 1), rtol=0, atol=1e-15)


# ----------------------------------------------------------------------------- joint limits, DC motor
def _limited(spec, limited, rng):
    import dataclasses
    return dataclasses.replace(spec, jnt_limited=np.asarray(limited, dtype=np.int32),
                               jnt_range=np.asarray(rng, dtype=np.float64).reshape(-1, 2))


def test_newton_with_limit_rows_matches_active_set_enumeration():
    """One-sided limit rows (J = +-e_d) and frictionless contacts are both one-sided
    quadratics D/2 min(x, 0)^2: the Newton optimum equals the solution of the linear
    system of the one active set that is self-consistent (brute force over all sets)."""
    rng = np.random.default_rng(21)
    for trial in range(30):
        nv, nc, nl = int(rng.integers(3, 7)), int(rng.integers(0, 3)), int(rng.integers(1, 4))
        M, a_s, J, aref, D, mu = random_problem(rng, nv, max(nc, 1), 0.0)
        if nc == 0:
            J, aref, D, mu = J[:0], aref[:0], D[:0], mu[:0]
        Jl = np.zeros((nl, nv))
        for l in range(nl):
            Jl[l, rng.integers(0, nv)] = rng.choice([-1.0, 1.0])
        arefl = rng.normal(size=nl) * 3
        Dl = rng.uniform(0.5, 5.0, nl)
        a, f, it, fl = Oracle.newton(M, a_s, J, aref, D, mu, Jl=Jl, arefl=arefl, Dl=Dl)
        rows = [(J[3 * c], aref[3 * c], D[3 * c]) for c in range(nc)] + list(zip(Jl, arefl, Dl))
        best = None
        for mask in range(1 << len(rows)):
            S = [i for i in range(len(rows)) if mask >> i & 1]
            H, rhs = M.copy(), M @ a_s
            for i in S:
                j, ar, d = rows[i]
                H += d * np.outer(j, j)
                rhs += d * ar * j
            x = np.linalg.solve(H, rhs)
            r = [rows[i][0] @ x - rows[i][1] for i in range(len(rows))]
            if all(r[i] <= 1e-12 for i in S) and all(r[i] >= -1e-12 for i in range(len(rows)) if i not in S):
                best = x
        assert best is not None
        np.testing.assert_allclose(a, best, rtol=1e-10, atol=1e-10)
        # limit forces: f = -D min(x, 0) >= 0 and stationarity M (a - a_s) = J^T f + Jl^T fl
        assert np.all(fl >= 0)
        np.testing.assert_allclose(M @ (a - a_s), J.T @ f + Jl.T @ fl, atol=1e-9 * max(1, np.abs(fl).max()))


def _impedance(r, solimp=(0.9, 0.95, 0.001, 0.5, 2.0)):
    """solimp d(r) (dmin, dmax, width, midpoint, power), restated from its definition."""
    d0, d1, width, mid, p = solimp
    x = abs(r) / width
    if x >= 1:
        return d1
    y = x ** p / mid ** (p - 1) if x <= mid else 1 - (1 - x) ** p / (1 - mid) ** (p - 1)
    return d0 + y * (d1 - d0)


def test_pendulum_resting_on_its_lower_limit():
    """A 1-link pendulum released above its lower limit lo = 0.5 rad falls onto it and
    settles where the limit force balances gravity: with J = e_d, at rest
    aref = -k d(r) r, D = d I / (1 - d) (A = 1/I for one dof), so the equilibrium r < 0
    solves  -d(r)^2 I k r / (1 - d(r)) = m g (L/2) sin(lo + r)  (k = 1/(dmax tc)^2, tc = 0.02)."""
    from scipy.optimize import brentq
    m, L, rad = 1.0, 0.3, 0.02
    spec = _limited(I.pendulum(1, noise=0.0), [1], [[0.5, 2.5]])
    Ip = m * (3 * rad ** 2 + L ** 2) / 12 + m * (L / 2) ** 2
    k = 1 / (0.95 * 0.02) ** 2
    fn = lambda r: -_impedance(r) ** 2 * Ip * k * r / (1 - _impedance(r)) - m * 9.81 * (L / 2) * math.sin(0.5 + r)
    r_star = brentq(fn, -0.2, -1e-12, xtol=1e-15)
    o = Oracle(spec)
    q, v, a = np.array([0.55]), np.zeros(1), np.zeros(1)
    for _ in range(1500):
        out = o.step(q, v, a, None)
        q, v, a = out["qpos"], out["qvel"], out["qacc"]
    assert abs(v[0]) < 1e-9
    assert abs(q[0] - (0.5 + r_star)) < 1e-9, (q[0] - 0.5, r_star)
    lim = o.limits(q, v)
    assert lim["nl"] == 1 and lim["sign"][0] == 1 and lim["dof"][0] == 0
    # the same pendulum with the limit on the other side: mirror image
    spec2 = _limited(I.pendulum(1, noise=0.0), [1], [[-2.5, -0.5]])
    o2 = Oracle(spec2)
    q, v, a = np.array([-0.55]), np.zeros(1), np.zeros(1)
    for _ in range(1500):
        out = o2.step(q, v, a, None)
        q, v, a = out["qpos"], out["qvel"], out["qacc"]
    assert abs(q[0] + 0.5 + r_star) < 1e-9
    assert o2.limits(q, v)["sign"][0] == -1


def test_dc_motor_follows_its_torque_speed_line():
    """A DC motor (stall torque ts = 2 N m, no-load speed w0 = 10 rad/s, torque limit
    tl = 1 N m) driving a free hinge inertia I (gravity off) with a far target: torque
    tl until w reaches w_k = w0 (1 - tl/ts), then ts (1 - w/w0), so
    w(t) = tl t / I for t <= t_k = I w_k / tl and w0 - (w0 - w_k) exp(-ts (t - t_k)/(I w0))
    after; semi-implicit Euler is exact on the first leg and O(h) on the second. The
    opposite target gives the mirror image; no torque beyond the no-load speed."""
    import dataclasses
    m, L, rad, h = 1.0, 0.3, 0.02, 0.001
    base = I.pendulum(1, noise=0.0, timestep=h, gravity=(0.0, 0.0, 0.0))
    spec = dataclasses.replace(base, act_jnt=np.array([0], dtype=np.int32), act_kp=np.array([1e4]),
                               act_kd=np.array([0.0]), act_dcmotor=np.array([[2.0, 10.0, 1.0]]))
    Ip = m * (3 * rad ** 2 + L ** 2) / 12 + m * (L / 2) ** 2
    o = Oracle(spec)
    ts, w0, tl = 2.0, 10.0, 1.0
    wk = w0 * (1 - tl / ts)
    tk = Ip * wk / tl
    for sgn in (1.0, -1.0):
        q, v, a = np.zeros(1), np.zeros(1), np.zeros(1)
        for n in range(1, 1201):
            out = o.step(q, v, a, np.array([sgn * 1e3]))
            q, v, a = out["qpos"], out["qvel"], out["qacc"]
            t = n * h
            if n == 100:
                assert abs(v[0] - sgn * tl * t / Ip) < 1e-9
            if t > tk + 0.1 and n % 100 == 0:
                w = w0 - (w0 - wk) * math.exp(-ts * (t - tk) / (Ip * w0))
                assert abs(v[0] - sgn * w) < 20 * h * (w0 - wk) / (Ip * w0 / ts) + 2e-2, (t, v[0], w)
        assert abs(v[0]) < w0
    # beyond the no-load speed the motor gives no driving torque, only braking up to tl
    q, v, a = np.zeros(1), np.array([12.0]), np.zeros(1)
    out = o.step(q, v, a, np.array([1e3]))
    assert abs(out["qacc"][0]) < 1e-12
    out = o.step(q, v, a, np.array([-1e3]))
    assert abs(out["qacc"][0] + tl / Ip) < 1e-9
