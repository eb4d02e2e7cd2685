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


def _hfield_box_spec(Z, half, box_half):
    spec0 = I.free_body(I.BOX, box_half, mass=1.0, pos=(0, 0, 0.3))
    gt = spec0.geom_type.copy()
    gt[0] = I.HFIELD
    return dataclasses.replace(spec0, geom_type=gt, hfield_data=Z, hfield_size=(half, half))


def test_spike_under_a_box_face_gives_one_contact_at_the_spike():
    """A flat grid with one raised vertex (3 cm) under the middle of a box whose bottom
    face hovers 1 cm above the ground: no box vertex is below the surface, the spike is
    2 cm inside the box, closest to the bottom face -> one contact, depth -0.02, normal +z,
    at the midpoint between the spike and the bottom face."""
    Z = np.zeros((41, 41))
    Z[20, 20] = 0.03                       # the vertex at (0, 0) on a 0.05 m grid
    spec = _hfield_box_spec(Z, 1.0, (0.1, 0.08, 0.05))
    o = Oracle(spec)
    q = spec.qpos_reset.copy()
    q[0:3] = [0.0, 0.0, 0.06]              # bottom face at z = 0.01
    q[3:7] = [1, 0, 0, 0]
    con = o.collide(q)
    assert con.shape[0] == 1
    np.testing.assert_allclose(con[0, 4], -0.02, atol=1e-14)
    np.testing.assert_allclose(con[0, 5:8], [0.0, 0.0, 0.02], atol=1e-14)
    np.testing.assert_allclose(con[0, 8:11], [0.0, 0.0, 1.0], atol=1e-14)
    q[2] = 0.085                           # bottom face above the spike: no contact
    assert o.collide(q).shape[0] == 0


def _quat_to_R(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _brute_box_contacts(Z, half, c, R, h):
    """Every candidate of the box-heightfield reading, by brute force over the whole grid:
    box vertices below the triangle under them, convex interior grid vertices inside the
    box; the 4 deepest (ties: vertices, then grid row-major) as (depth, pos, normal) in
    candidate order."""
    nrow, ncol = Z.shape
    dx, dy = 2 * half / (ncol - 1), 2 * half / (nrow - 1)
    cand = []
    for v in range(8):
        loc = np.array([(1 if v & 1 else -1) * h[0], (1 if v & 2 else -1) * h[1], (1 if v & 4 else -1) * h[2]])
        p = c + R @ loc
        u, w = (p[0] + half) / dx, (p[1] + half) / dy
        if not (0 <= u <= ncol - 1 and 0 <= w <= nrow - 1):
            continue
        j, i = min(int(u), ncol - 2), min(int(w), nrow - 2)
        a = np.array([-half + j * dx, -half + i * dy, Z[i, j]])
        b10 = np.array([-half + (j + 1) * dx, -half + i * dy, Z[i, j + 1]])
        b11 = np.array([-half + (j + 1) * dx, -half + (i + 1) * dy, Z[i + 1, j + 1]])
        b01 = np.array([-half + j * dx, -half + (i + 1) * dy, Z[i + 1, j]])
        B, Cc = (b11, b01) if (w - i) > (u - j) else (b10, b11)
        n = np.cross(B - a, Cc - a)
        n /= np.linalg.norm(n)
        d = float(n @ (p - a))
        if d < 0:
            cand.append((d, v, p - n * 0.5 * d, n))
    for i in range(1, nrow - 1):
        for j in range(1, ncol - 1):
            if not Z[i, j] - 0.25 * ((Z[i - 1, j] + Z[i + 1, j]) + (Z[i, j - 1] + Z[i, j + 1])) > 1e-9:
                continue
            g = np.array([-half + j * dx, -half + i * dy, Z[i, j]])
            p = R.T @ (g - c)
            if not np.all(np.abs(p) < h):
                continue
            dist = h - np.abs(p)
            k = int(np.argmin(dist))
            nl = np.zeros(3)
            nl[k] = -1.0 if p[k] >= 0 else 1.0
            n = R @ nl
            cand.append((-dist[k], 8 + i * ncol + j, g + n * 0.5 * -dist[k], n))
    cand.sort(key=lambda x: (x[0], x[1]))
    return sorted(cand[:4], key=lambda x: x[1])


def test_box_on_bumps_matches_brute_force_candidates():
    """Random box poses over Gaussian bumps: the oracle's contacts (footprint-limited
    search) equal the brute-force candidates over the whole grid, and some contacts come
    from grid vertices pressing into a box face."""
    terrain = I.with_terrain(I.quadruped(), nrow=41, ncol=41, half=1.0, amplitude=0.12, seed=7).hfield_data
    h = np.array([0.12, 0.07, 0.04])
    spec = _hfield_box_spec(terrain, 1.0, tuple(h))
    o = Oracle(spec)
    rng = np.random.default_rng(11)
    xs = np.linspace(-1, 1, 41)
    grid_contacts = total = 0
    for _ in range(150):
        q = spec.qpos_reset.copy()
        q[0:2] = rng.uniform(-0.7, 0.7, 2)
        zs = float(np.interp(q[1], xs, [np.interp(q[0], xs, row) for row in terrain]))
        q[2] = zs + rng.uniform(-0.02, 0.06)
        qq = rng.normal(size=4) * np.array([4.0, 0.3, 0.3, 1.0])   # mostly yaw
        q[3:7] = qq / np.linalg.norm(qq)
        con = o.collide(q)
        ref = _brute_box_contacts(terrain, 1.0, q[0:3], _quat_to_R(q[3:7]), h)
        assert len(con) == len(ref)
        for row, (d, key, pos, n) in zip(con, ref):
            np.testing.assert_allclose(row[4], d, atol=1e-12)
            np.testing.assert_allclose(row[5:8], pos, atol=1e-12)
            np.testing.assert_allclose(row[8:11], n, atol=1e-12)
            grid_contacts += key >= 8
        total += len(con)
    assert total > 100 and grid_contacts > 10
