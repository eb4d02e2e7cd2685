"""Pins of the oracle's box-box narrow phase: closed-form resting and edge-edge
configurations, the separating-axis minimum against brute-force direction
sampling, every manifold point inside both boxes, and force balance of a cube
resting on a table box."""
import itertools
import math

import numpy as np

from oracle import Oracle
from paper_2601_22074_b300 import inputs as I


def rot(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def random_rot(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_cube_resting_on_table_closed_form():
    hA, hB = np.array([0.4, 0.4, 0.2]), np.array([0.025] * 3)
    cA = np.array([0.45, 0.0, 0.2])
    delta = 3e-4
    for yaw in (0.0, 0.5):
        R = rot([0, 0, 1], yaw)
        cB = np.array([0.5, 0.1, 0.4 + 0.025 - delta])
        con, axis, _ = Oracle.box_box(cA, np.eye(3), hA, cB, R, hB)
        assert axis == 2 and len(con) == 4
        corners = np.array([cB + R @ (np.array([sx, sy, -1]) * hB)
                            for sx, sy in itertools.product((-1, 1), repeat=2)])
        got = con[:, 5:8]
        for c in corners:
            k = np.argmin(np.linalg.norm(got[:, :2] - c[:2], axis=1))
            np.testing.assert_allclose(got[k], [c[0], c[1], 0.4 - delta / 2], atol=1e-12)
        np.testing.assert_allclose(con[:, 4], -delta, atol=1e-12)
        np.testing.assert_allclose(con[:, 8:11], np.tile([0, 0, 1.0], (4, 1)), atol=1e-12)


def test_edge_edge_closed_form():
    h = 0.5
    RA, RB = rot([0, 1, 0], math.pi / 4), rot([1, 0, 0], math.pi / 4)
    zB = 2 * h * math.sqrt(2) - 0.01
    con, axis, minov = Oracle.box_box(np.zeros(3), RA, np.full(3, h), np.array([0, 0, zB]), RB, np.full(3, h))
    assert axis >= 6 and len(con) == 1
    np.testing.assert_allclose(con[0, 4], -0.01, atol=1e-12)
    np.testing.assert_allclose(con[0, 5:8], [0, 0, zB / 2], atol=1e-12)
    np.testing.assert_allclose(con[0, 8:11], [0, 0, 1], atol=1e-12)


def sampled_min_overlap(cA, RA, hA, cB, RB, hB, n=40000, seed=0):
    """Brute force over directions: dense random sample, then a shrinking random local
    search around the best few directions."""
    rng = np.random.default_rng(seed)

    def ov(L):
        L = L / np.linalg.norm(L, axis=-1, keepdims=True)
        return np.abs(L @ RA) @ hA + np.abs(L @ RB) @ hB - np.abs(L @ (cB - cA))

    L = rng.normal(size=(n, 3))
    vals = ov(L)
    starts = L[np.argsort(vals)[:8]]
    best = float(vals.min())
    for x in starts:
        x = x / np.linalg.norm(x)
        f = float(ov(x[None])[0])
        sig = 0.05
        for _ in range(400):
            cand = x + sig * rng.normal(size=(64, 3))
            v = ov(cand)
            k = int(np.argmin(v))
            if v[k] < f:
                f, x = float(v[k]), cand[k] / np.linalg.norm(cand[k])
            else:
                sig *= 0.85
        best = min(best, f)
    return best


def test_separating_axis_minimum_against_direction_sampling():
    rng = np.random.default_rng(3)
    checked = 0
    for _ in range(30):
        hA, hB = rng.uniform(0.05, 0.3, 3), rng.uniform(0.05, 0.3, 3)
        RA, RB = random_rot(rng), random_rot(rng)
        cA = np.zeros(3)
        cB = rng.normal(size=3) * 0.3
        con, axis, minov = Oracle.box_box(cA, RA, hA, cB, RB, hB)
        samp = sampled_min_overlap(cA, RA, hA, cB, RB, hB)
        if axis < 0:
            # separated: the reported separating axis is one direction of the search space
            assert len(con) == 0 and minov < 0 and samp <= minov + 1e-12
        else:
            # overlapping: the 15 axes contain the minimiser of the overlap over all
            # directions, so sampling can only find larger overlaps, and finds this one
            checked += 1
            assert minov >= 0
            assert samp >= minov - 1e-12
            assert samp <= minov + 1e-6 * (hA.sum() + hB.sum())
    assert checked > 10


def test_manifold_points_lie_in_both_boxes():
    rng = np.random.default_rng(4)
    n = 0
    for _ in range(200):
        hA, hB = rng.uniform(0.05, 0.3, 3), rng.uniform(0.05, 0.3, 3)
        RA, RB = random_rot(rng), random_rot(rng)
        cA, cB = np.zeros(3), rng.normal(size=3) * 0.25
        con, axis, _ = Oracle.box_box(cA, RA, hA, cB, RB, hB)
        for c in con:
            p, dist, nrm = c[5:8], c[4], c[8:11]
            assert dist <= 0
            assert abs(np.linalg.norm(nrm) - 1) < 1e-12
            for cc, R, h in ((cA, RA, hA), (cB, RB, hB)):
                loc = R.T @ (p - cc)
                assert np.all(np.abs(loc) <= h + abs(dist) + 1e-9)
            n += 1
    assert n > 50


def _cube_on_table_spec():
    b = I._Builder("cube_table")
    b.geom(0, I.BOX, (0.4, 0.4, 0.2), pos=(0.45, 0, 0.2), contype=2, conaffinity=1)
    cube = b.body(0, (0.45, 0.0, 0.425), mass=0.1, inertia=I.box_inertia(0.1, (0.025,) * 3))
    b.joint(cube, I.FREE)
    b.geom(cube, I.BOX, (0.025,) * 3, contype=1, conaffinity=2)
    return b.build(I.Options(timestep=0.005))


def test_cube_resting_on_table_force_balance():
    spec = _cube_on_table_spec()
    o = Oracle(spec)
    q, v, a = spec.qpos_reset.copy(), np.zeros(6), np.zeros(6)
    for _ in range(300):
        r = o.step(q, v, a, None, want_contacts=True)
        q, v, a = r["qpos"], r["qvel"], r["qacc"]
    con = r["contacts"]
    assert len(con) == 4
    np.testing.assert_allclose(con[:, 18].sum(), 0.1 * 9.81, rtol=1e-8)
    assert np.abs(con[:, 19:21]).max() < 1e-8
    np.testing.assert_allclose(-con[:, 4] * 1e3, 0.367182, rtol=2e-4)  # same penetration fixed point
