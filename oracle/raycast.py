"""Ray casting against the model's primitives, FP64 (TEST INFRASTRUCTURE ONLY).

The ray-cast sensor of the paper's components (section "Components": ray casts from a
body, distance per ray) restated from the definitions: a ray o + t d (t >= 0, unit d)
and the first t at which it enters a solid -- a plane's lower half-space, a sphere, a
capsule (the set of points within r of a segment of half-length h along the geom's z
axis), a box (|x_i| <= h_i in the geom frame), a heightfield (below its triangulated
elevation grid: the first triangle the ray meets, every triangle tested); 0 for an origin
inside a solid. Geom poses come from the oracle's forward kinematics.
"""
from __future__ import annotations

import math

import numpy as np

PLANE, SPHERE, CAPSULE, BOX, HFIELD = 0, 1, 2, 3, 4


def _sphere(o, d, c, r):
    p = o - c
    b = p @ d
    cc = p @ p - r * r
    if cc <= 0:
        return 0.0
    disc = b * b - cc
    if disc < 0 or b > 0:
        return math.inf
    return -b - math.sqrt(disc)


def ray_primitive(gtype, size, o, d) -> float:
    """First hit distance of a ray given in the primitive's own frame."""
    o = np.asarray(o, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    if gtype == PLANE:
        if o[2] <= 0:
            return 0.0
        return -o[2] / d[2] if d[2] < 0 else math.inf
    if gtype == SPHERE:
        return _sphere(o, d, np.zeros(3), size[0])
    if gtype == CAPSULE:
        r, h = size[0], size[1]
        zc = min(max(o[2], -h), h)
        if o[0] ** 2 + o[1] ** 2 + (o[2] - zc) ** 2 <= r * r:
            return 0.0
        best = math.inf
        a = d[0] ** 2 + d[1] ** 2
        if a > 1e-24:
            b = o[0] * d[0] + o[1] * d[1]
            c = o[0] ** 2 + o[1] ** 2 - r * r
            disc = b * b - a * c
            if disc >= 0:
                t = (-b - math.sqrt(disc)) / a
                if t >= 0 and abs(o[2] + t * d[2]) <= h:
                    best = t
        best = min(best, _sphere(o, d, np.array([0, 0, h]), r), _sphere(o, d, np.array([0, 0, -h]), r))
        return best
    tmin, tmax = 0.0, math.inf
    for i in range(3):
        if abs(d[i]) < 1e-24:
            if abs(o[i]) > size[i]:
                return math.inf
        else:
            t1, t2 = (-size[i] - o[i]) / d[i], (size[i] - o[i]) / d[i]
            tmin, tmax = max(tmin, min(t1, t2)), min(tmax, max(t1, t2))
    return tmin if tmax >= tmin else math.inf


def hfield_triangles(spec):
    """[ntri, 3, 3] triangle vertices of the model's elevation grid (geom frame)."""
    Z = np.asarray(spec.hfield_data, dtype=np.float64)
    nrow, ncol = Z.shape
    hx, hy = spec.hfield_size
    xs = np.linspace(-hx, hx, ncol)
    ys = np.linspace(-hy, hy, nrow)
    tris = []
    for i in range(nrow - 1):
        for j in range(ncol - 1):
            v00 = (xs[j], ys[i], Z[i, j])
            v10 = (xs[j + 1], ys[i], Z[i, j + 1])
            v11 = (xs[j + 1], ys[i + 1], Z[i + 1, j + 1])
            v01 = (xs[j], ys[i + 1], Z[i + 1, j])
            tris.append((v00, v10, v11))
            tris.append((v00, v11, v01))
    return np.array(tris)


def surface_height(spec, x, y):
    """Elevation of the triangulated grid at (x, y), None outside it."""
    Z = np.asarray(spec.hfield_data, dtype=np.float64)
    nrow, ncol = Z.shape
    hx, hy = spec.hfield_size
    dx, dy = 2 * hx / (ncol - 1), 2 * hy / (nrow - 1)
    u, v = (x + hx) / dx, (y + hy) / dy
    if u < 0 or v < 0 or u > ncol - 1 or v > nrow - 1:
        return None
    j, i = min(int(u), ncol - 2), min(int(v), nrow - 2)
    fu, fv = u - j, v - i
    z00, z10, z11, z01 = Z[i, j], Z[i, j + 1], Z[i + 1, j + 1], Z[i + 1, j]
    if fv > fu:    # triangle (v00, v11, v01)
        return z00 + fu * (z11 - z01) + fv * (z01 - z00)
    return z00 + fu * (z10 - z00) + fv * (z11 - z10)


def ray_hfield(spec, tris, o, d) -> float:
    zs = surface_height(spec, o[0], o[1])
    if zs is not None and o[2] <= zs:
        return 0.0
    a, b, c = tris[:, 0], tris[:, 1], tris[:, 2]
    e1, e2 = b - a, c - a
    pv = np.cross(d[None], e2)
    det = np.einsum("ij,ij->i", e1, pv)
    ok = np.abs(det) > 1e-15
    inv = np.where(ok, 1.0 / np.where(ok, det, 1.0), 0.0)
    tv = o[None] - a
    u = np.einsum("ij,ij->i", tv, pv) * inv
    qv = np.cross(tv, e1)
    v = (qv @ d) * inv
    t = np.einsum("ij,ij->i", e2, qv) * inv
    hit = ok & (u >= 0) & (u <= 1) & (v >= 0) & (u + v <= 1) & (t >= 0)
    return float(t[hit].min()) if np.any(hit) else math.inf


def raycast(o_model, spec, qpos, body, origins, directions, max_dist, world_only=True) -> np.ndarray:
    f = o_model.fk(qpos)
    Rb, xb = f["xmat"][body], f["xpos"][body]
    tris = hfield_triangles(spec) if getattr(spec, "hfield_data", None) is not None else None
    out = np.full(len(origins), float(max_dist))
    for r, (ob, db) in enumerate(zip(np.asarray(origins, float), np.asarray(directions, float))):
        o = xb + Rb @ ob
        d = Rb @ db
        for g in range(spec.ngeom):
            gb = int(spec.geom_body[g])
            if (gb != 0) if world_only else (gb == body):
                continue
            c, R = f["gxpos"][g], f["gxmat"][g]
            if int(spec.geom_type[g]) == HFIELD:
                t = ray_hfield(spec, tris, R.T @ (o - c), R.T @ d)
            else:
                t = ray_primitive(int(spec.geom_type[g]), spec.geom_size[g], R.T @ (o - c), R.T @ d)
            out[r] = min(out[r], t)
    return out
