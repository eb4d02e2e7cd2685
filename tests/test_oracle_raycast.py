"""Pins of the oracle's ray casts (CPU): hand-computed hits and ray marching along the
primitives' signed-distance functions (textbook closed forms, independent of the
intersection formulas)."""
import math

import numpy as np

from oracle import raycast as RC


def sdf(gtype, size, p):
    p = np.asarray(p, dtype=np.float64)
    if gtype == RC.PLANE:
        return p[2]
    if gtype == RC.SPHERE:
        return np.linalg.norm(p) - size[0]
    if gtype == RC.CAPSULE:
        q = p.copy()
        q[2] -= min(max(p[2], -size[1]), size[1])
        return np.linalg.norm(q) - size[0]
    q = np.abs(p) - np.asarray(size[:3])
    return np.linalg.norm(np.maximum(q, 0.0)) + min(max(q[0], q[1], q[2]), 0.0)


def march(gtype, size, o, d, tmax=3.0):
    """Sphere tracing: step by the SDF (never past the surface) to the first crossing."""
    t = 0.0
    if sdf(gtype, size, o) <= 0:
        return 0.0
    for _ in range(20000):
        s = sdf(gtype, size, o + t * d)
        if s < 1e-10:
            return t
        t += s
        if t > tmax:
            return math.inf
    return t


def test_hand_computed_hits():
    down = np.array([0.0, 0.0, -1.0])
    assert RC.ray_primitive(RC.PLANE, [0, 0, 0], [0.3, 0.2, 0.7], down) == 0.7
    assert RC.ray_primitive(RC.PLANE, [0, 0, 0], [0, 0, 0.7], -down) == math.inf
    assert abs(RC.ray_primitive(RC.SPHERE, [0.2, 0, 0], [-1.0, 0, 0], [1.0, 0, 0]) - 0.8) < 1e-15
    assert abs(RC.ray_primitive(RC.BOX, [0.1, 0.2, 0.3], [0, 0, 1.0], down) - 0.7) < 1e-15
    assert abs(RC.ray_primitive(RC.CAPSULE, [0.05, 0.2, 0], [1.0, 0, 0.1], [-1.0, 0, 0]) - 0.95) < 1e-15
    assert abs(RC.ray_primitive(RC.CAPSULE, [0.05, 0.2, 0], [0, 0, 1.0], down) - 0.75) < 1e-15   # cap
    assert RC.ray_primitive(RC.BOX, [0.1, 0.1, 0.1], [0.05, 0, 0], down) == 0.0                  # inside


def test_intersections_match_sphere_tracing():
    rng = np.random.default_rng(8)
    for gtype, size in ((RC.SPHERE, [0.3, 0, 0]), (RC.CAPSULE, [0.1, 0.25, 0]), (RC.BOX, [0.2, 0.1, 0.3]),
                        (RC.PLANE, [0, 0, 0])):
        hits = 0
        for _ in range(200):
            o = rng.uniform(-1, 1, 3)
            target = rng.normal(0, 0.2, 3)
            d = target - o
            d /= np.linalg.norm(d)
            t = RC.ray_primitive(gtype, size, o, d)
            tm = march(gtype, size, o, d)
            if math.isinf(tm):
                assert math.isinf(t) or t > 3.0, (gtype, o, d, t)
            else:
                hits += 1
                assert abs(t - tm) < 1e-6, (gtype, o, d, t, tm)
        assert hits > 40


def test_heightfield_rays_match_height_marching():
    """Rays against a bumpy grid: the first t where the ray point drops below the
    interpolated surface, found by fine stepping, equals the triangle hit."""
    from paper_2601_22074_b300 import inputs as I
    spec = I.with_terrain(I.quadruped(), nrow=15, ncol=15, half=1.0, amplitude=0.2, seed=3)
    tris = RC.hfield_triangles(spec)
    rng = np.random.default_rng(9)
    hits = 0
    for _ in range(60):
        o = np.array([rng.uniform(-0.8, 0.8), rng.uniform(-0.8, 0.8), rng.uniform(0.2, 0.6)])
        d = np.array([rng.normal(0, 0.5), rng.normal(0, 0.5), -1.0])
        d /= np.linalg.norm(d)
        t = RC.ray_hfield(spec, tris, o, d)
        tm = math.inf
        for k in range(1, 40001):
            s = k * 5e-5
            p = o + s * d
            zs = RC.surface_height(spec, p[0], p[1])
            if zs is None:
                break
            if p[2] <= zs:
                tm = s
                break
        if math.isinf(tm):
            assert math.isinf(t) or t > (k - 1) * 5e-5 - 1e-9
        else:
            hits += 1
            assert tm - 5e-5 - 1e-9 <= t <= tm + 1e-9, (t, tm)
    assert hits > 30


def _sdf_grad(gtype, size, p, h=1e-6):
    g = np.array([(sdf(gtype, size, p + h * e) - sdf(gtype, size, p - h * e)) / (2 * h) for e in np.eye(3)])
    return g / np.linalg.norm(g)


def test_normals_are_the_signed_distance_gradient_at_the_hit():
    """At every hit the oracle's normal equals the normalised central-difference gradient
    of the primitive's signed-distance function (a closed form independent of the
    intersection formulas), faces the ray, and is zero for misses and inside origins."""
    rng = np.random.default_rng(12)
    for gtype, size in ((RC.SPHERE, [0.3, 0, 0]), (RC.CAPSULE, [0.1, 0.25, 0]), (RC.BOX, [0.2, 0.1, 0.3]),
                        (RC.PLANE, [0, 0, 0])):
        hits = 0
        for _ in range(200):
            o = rng.uniform(-1, 1, 3)
            d = rng.normal(0, 0.2, 3) - o
            d /= np.linalg.norm(d)
            t, n = RC.ray_primitive_n(gtype, size, o, d)
            if math.isinf(t) or t == 0.0:
                assert np.array_equal(n, np.zeros(3))
                continue
            hits += 1
            p = o + t * d
            g = _sdf_grad(gtype, size, p)
            np.testing.assert_allclose(n, g, atol=1e-5)
            assert n @ d < 0
        assert hits > 40
    t, n = RC.ray_primitive_n(RC.BOX, [0.1, 0.2, 0.3], [0.0, 0.0, 1.0], [0, 0, -1.0])
    assert np.array_equal(n, [0.0, 0.0, 1.0])                         # top face
    t, n = RC.ray_primitive_n(RC.BOX, [0.1, 0.1, 0.1], [0.05, 0, 0], [0, 0, -1.0])
    assert t == 0.0 and np.array_equal(n, np.zeros(3))                 # origin inside


def test_heightfield_normals_match_the_surface_gradient():
    from paper_2601_22074_b300 import inputs as I
    spec = I.with_terrain(I.quadruped(), nrow=15, ncol=15, half=1.0, amplitude=0.2, seed=3)
    tris = RC.hfield_triangles(spec)
    rng = np.random.default_rng(13)
    checked = 0
    for _ in range(60):
        o = np.array([rng.uniform(-0.8, 0.8), rng.uniform(-0.8, 0.8), 0.6])
        d = np.array([rng.normal(0, 0.3), rng.normal(0, 0.3), -1.0])
        d /= np.linalg.norm(d)
        t, n = RC.ray_hfield_n(spec, tris, o, d)
        if math.isinf(t):
            continue
        p = o + t * d
        # gradient of the interpolated surface from one-sided differences inside the
        # triangle (the hit point's cell); normal (-dh/dx, -dh/dy, 1) normalised
        h = 1e-7
        z0 = RC.surface_height(spec, p[0], p[1])
        cands = []
        for sx in (1, -1):
            for sy in (1, -1):
                zx = RC.surface_height(spec, p[0] + sx * h, p[1])
                zy = RC.surface_height(spec, p[0], p[1] + sy * h)
                if zx is None or zy is None:
                    continue
                g = np.array([-(zx - z0) / (sx * h), -(zy - z0) / (sy * h), 1.0])
                cands.append(g / np.linalg.norm(g))
        assert min(np.abs(c - n).max() for c in cands) < 1e-5, (n, cands)
        assert n[2] > 0
        checked += 1
    assert checked > 30
