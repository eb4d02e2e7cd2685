"""Ray casting against the model's primitives, FP64 (TEST INFRASTRUCTURE ONLY).

The ray-cast sensor of the paper's components (section "Components": ray casts from a
body returning per-ray distances, hit positions and surface normals) restated from the
definitions: a ray o + t d (t >= 0, unit d) and the first t at which it enters a solid --
a plane's lower half-space, a sphere, a capsule (the set of points within r of a segment
of half-length h along the geom's z axis), a box (|x_i| <= h_i in the geom frame), a
heightfield (below its triangulated elevation grid: the first triangle the ray meets,
every triangle tested); 0 for an origin inside a solid. Every geom is tested (no
acceleration structure). The normal is the outward unit normal of the solid at the entry
point (the plane's z axis; from the sphere centre or the capsule's segment; the box face
whose slab the ray enters last, the lower axis on ties; the upward normal of the hit
triangle), zero for a miss or an origin inside; among geoms hit at the same distance the
lowest geom index gives it. Geom poses come from the oracle's forward kinematics.
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


def ray_primitive_n(gtype, size, o, d):
    """(first hit distance, outward unit normal at the hit) of a ray in the primitive's own
    frame; the normal is zero for a miss or an origin inside."""
    o = np.asarray(o, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    zero = np.zeros(3)
    if gtype == PLANE:
        if o[2] <= 0:
            return 0.0, zero
        return (-o[2] / d[2], np.array([0.0, 0.0, 1.0])) if d[2] < 0 else (math.inf, zero)
    if gtype == SPHERE:
        t = _sphere(o, d, np.zeros(3), size[0])
        return t, ((o + t * d) / size[0] if 0 < t < math.inf else zero)
    if gtype == CAPSULE:
        r, h = size[0], size[1]
        zc = min(max(o[2], -h), h)
        if o[0] ** 2 + o[1] ** 2 + (o[2] - zc) ** 2 <= r * r:
            return 0.0, zero
        best, n = math.inf, zero
        a = d[0] ** 2 + d[1] ** 2
        if a > 1e-24:
            b = o[0] * d[0] + o[1] * d[1]
            c = o[0] ** 2 + o[1] ** 2 - r * r
            disc = b * b - a * c
            if disc >= 0:
                t = (-b - math.sqrt(disc)) / a
                if t >= 0 and abs(o[2] + t * d[2]) <= h:
                    p = o + t * d
                    best, n = t, np.array([p[0], p[1], 0.0]) / r
        for zc in (h, -h):
            cen = np.array([0.0, 0.0, zc])
            t = _sphere(o, d, cen, r)
            if t < best:
                best, n = t, (o + t * d - cen) / r
        return best, n
    tmin, tmax, axis, sgn = 0.0, math.inf, -1, 0.0
    for i in range(3):
        if abs(d[i]) < 1e-24:
            if abs(o[i]) > size[i]:
                return math.inf, zero
        else:
            t1, t2 = (-size[i] - o[i]) / d[i], (size[i] - o[i]) / d[i]
            if min(t1, t2) > tmin:
                tmin, axis, sgn = min(t1, t2), i, (-1.0 if t1 < t2 else 1.0)
            tmax = min(tmax, max(t1, t2))
    if not tmax >= tmin:
        return math.inf, zero
    n = zero.copy()
    if axis >= 0:
        n[axis] = sgn
    return tmin, n


def ray_primitive(gtype, size, o, d) -> float:
    """First hit distance of a ray given in the primitive's own frame."""
    return ray_primitive_n(gtype, size, o, d)[0]


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
    return ray_hfield_n(spec, tris, o, d)[0]


def ray_hfield_n(spec, tris, o, d):
    """(first hit, upward unit normal of the hit triangle) against the grid (geom frame)."""
    zs = surface_height(spec, o[0], o[1])
    if zs is not None and o[2] <= zs:
        return 0.0, np.zeros(3)
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
    if not np.any(hit):
        return math.inf, np.zeros(3)
    k = int(np.flatnonzero(hit)[np.argmin(t[hit])])
    n = np.cross(e1[k], e2[k])
    return float(t[k]), n / np.linalg.norm(n)


def raycast_hits(o_model, spec, qpos, body, origins, directions, max_dist, world_only=True):
    """(distances [nray], hit positions [nray, 3], normals [nray, 3]) of rays fixed to
    `body` (body-frame origins and unit directions); a miss reports max_dist, the point
    at max_dist and a zero normal."""
    f = o_model.fk(qpos)
    Rb, xb = f["xmat"][body], f["xpos"][body]
    tris = hfield_triangles(spec) if getattr(spec, "hfield_data", None) is not None else None
    n_ray = len(origins)
    dist = np.full(n_ray, float(max_dist))
    pos = np.zeros((n_ray, 3))
    nrm = np.zeros((n_ray, 3))
    for r, (ob, db) in enumerate(zip(np.asarray(origins, float), np.asarray(directions, float))):
        o = xb + Rb @ ob
        d = Rb @ db
        for g in range(spec.ngeom):
            gb = int(spec.geom_body[g])
            if (gb != 0) if world_only else (gb == body):
                continue
            c, R = f["gxpos"][g], f["gxmat"][g]
            if int(spec.geom_type[g]) == HFIELD:
                t, n = ray_hfield_n(spec, tris, R.T @ (o - c), R.T @ d)
            else:
                t, n = ray_primitive_n(int(spec.geom_type[g]), spec.geom_size[g], R.T @ (o - c), R.T @ d)
            if t < dist[r]:              # strict: the lowest geom index keeps a tie
                dist[r], nrm[r] = t, R @ n
        pos[r] = o + dist[r] * d
    return dist, pos, nrm


def raycast(o_model, spec, qpos, body, origins, directions, max_dist, world_only=True) -> np.ndarray:
    return raycast_hits(o_model, spec, qpos, body, origins, directions, max_dist, world_only)[0]
