"""Pins of the oracle's heightfield contacts (CPU): a flat grid reproduces the plane, a
planar tilted grid reproduces a tilted plane geom, and on bumps the sphere contact
distance equals brute-force sampling of the triangulated surface."""
import dataclasses
import math

import numpy as np

from oracle import Oracle
from paper_2601_22074_b300 import inputs as I


def test_flat_heightfield_reproduces_the_plane():
    for base, ctrl_of in ((I.quadruped(), True), (I.humanoid(), True)):
        flat = I.with_terrain(base, amplitude=0.0)
        runs = []
        for spec in (base, flat):
            o = Oracle(spec)
            q, v = o.reset(0, 3)
            a = np.zeros(spec.nv)
            u = spec.qpos_reset[spec.act_qposadr()]
            for _ in range(40):
                r = o.step(q, v, a, u, nsub=4, want_contacts=True)
                q, v, a = r["qpos"], r["qvel"], r["qacc"]
            runs.append((q, r["contacts"]))
        # the same trajectory up to the rounding of the grid-frame transforms
        np.testing.assert_allclose(runs[0][0], runs[1][0], atol=1e-10)
        np.testing.assert_allclose(runs[0][1], runs[1][1], atol=1e-9)
        assert len(runs[0][1]) > 0


def _tilted(a, b, half=1.0, n=9):
    xs = np.linspace(-half, half, n)
    X, Y = np.meshgrid(xs, xs)
    return a * X + b * Y


def test_planar_heightfield_matches_a_tilted_plane():
    a, b = 0.2, -0.1
    nrm = np.array([-a, -b, 1.0]) / math.sqrt(a * a + b * b + 1)
    # quaternion taking z to nrm
    ax = np.cross([0, 0, 1.0], nrm)
    ang = math.acos(nrm[2])
    quat = np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * ax / np.linalg.norm(ax)])
    rng = np.random.default_rng(2)
    for gtype, size in ((I.SPHERE, (0.1,)), (I.BOX, (0.1, 0.08, 0.05)), (I.CAPSULE, (0.05, 0.1))):
        spec = I.free_body(gtype, size, mass=1.0, pos=(0, 0, 0.3))
        gq = spec.geom_quat.copy()
        gq[0] = quat
        plane = dataclasses.replace(spec, geom_quat=gq)
        gt = spec.geom_type.copy()
        gt[0] = I.HFIELD
        hf = dataclasses.replace(spec, geom_type=gt, hfield_data=_tilted(a, b), hfield_size=(1.0, 1.0))
        op, oh = Oracle(plane), Oracle(hf)
        found = 0
        for _ in range(40):
            q = spec.qpos_reset.copy()
            q[0:2] = rng.uniform(-0.5, 0.5, 2)
            q[2] = a * q[0] + b * q[1] + rng.uniform(-0.05, 0.15)
            qq = rng.normal(size=4)
            q[3:7] = qq / np.linalg.norm(qq)
            cp, ch = op.collide(q), oh.collide(q)
            assert len(cp) == len(ch)
            if len(cp):
                found += 1
                np.testing.assert_allclose(ch[:, 4:17], cp[:, 4:17], atol=1e-12)
        assert found > 5


def _surface_distance(spec, c, rad, samples=60):
    """Brute force: the smallest distance from c to points sampled on every triangle near
    the sphere's footprint."""
    Z = spec.hfield_data
    nrow, ncol = Z.shape
    hx, hy = spec.hfield_size
    xs = np.linspace(-hx, hx, ncol)
    ys = np.linspace(-hy, hy, nrow)
    best = math.inf
    u = np.linspace(0, 1, samples)
    U, V = np.meshgrid(u, u)
    keep = U + V <= 1
    U, V = U[keep], V[keep]
    for i in range(nrow - 1):
        for j in range(ncol - 1):
            if abs(xs[j] - c[0]) > rad + 0.2 or abs(ys[i] - c[1]) > rad + 0.2:
                continue
            v00 = np.array([xs[j], ys[i], Z[i, j]])
            v10 = np.array([xs[j + 1], ys[i], Z[i, j + 1]])
            v11 = np.array([xs[j + 1], ys[i + 1], Z[i + 1, j + 1]])
            v01 = np.array([xs[j], ys[i + 1], Z[i + 1, j]])
            for A, B, Cc in ((v00, v10, v11), (v00, v11, v01)):
                P = A[None] + U[:, None] * (B - A)[None] + V[:, None] * (Cc - A)[None]
                best = min(best, np.linalg.norm(P - c[None], axis=1).min())
    return best


def test_sphere_on_bumps_matches_surface_sampling():
    spec0 = I.free_body(I.SPHERE, (0.08,), mass=1.0, pos=(0, 0, 0.3))
    gt = spec0.geom_type.copy()
    gt[0] = I.HFIELD
    terrain = I.with_terrain(I.quadruped(), nrow=21, ncol=21, half=1.0, amplitude=0.15, seed=4).hfield_data
    spec = dataclasses.replace(spec0, geom_type=gt, hfield_data=terrain, hfield_size=(1.0, 1.0))
    o = Oracle(spec)
    rng = np.random.default_rng(6)
    checked = 0
    for _ in range(60):
        q = spec.qpos_reset.copy()
        q[0:2] = rng.uniform(-0.7, 0.7, 2)
        # height: surface under the centre + something within the radius (above the surface)
        xs = np.linspace(-1, 1, 21)
        zs = float(np.interp(q[1], xs, [np.interp(q[0], xs, row) for row in terrain]))
        q[2] = zs + rng.uniform(0.0, 0.1)
        con = o.collide(q)
        d = _surface_distance(spec, q[0:3], 0.08) - 0.08
        if len(con):
            checked += 1
            assert abs(con[0, 4] - d) < 2e-3, (con[0, 4], d)
        else:
            assert d > -1e-3
    assert checked > 10
