"""Pins of the oracle's observation terms and contact-sensor bookkeeping (CPU):
closed-form rotations, scipy's rotation routine, force balance of a resting box, and a
hand-worked air-time sequence."""
import math

import numpy as np
from scipy.spatial.transform import Rotation

from oracle import Oracle
from oracle import sensors as S
from paper_2601_22074_b300 import inputs as I


def test_quaternion_matrix_matches_closed_forms_and_scipy():
    th = 0.7
    qz = [math.cos(th / 2), 0, 0, math.sin(th / 2)]
    np.testing.assert_allclose(S.quat_to_matrix(qz), [[math.cos(th), -math.sin(th), 0],
                                                      [math.sin(th), math.cos(th), 0], [0, 0, 1]], atol=1e-15)
    rng = np.random.default_rng(0)
    for _ in range(20):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()   # scipy: (x, y, z, w)
        np.testing.assert_allclose(S.quat_to_matrix(q), ref, atol=1e-12)


def test_observation_terms_of_a_tilted_and_turned_base():
    spec = I.quadruped()
    q = spec.qpos_reset.copy()
    v = np.zeros(spec.nv)
    obs = S.observe(spec, q, v, None)
    np.testing.assert_allclose(obs[0:3], [0, 0, -1], atol=1e-15)          # upright
    th = 0.3                                                             # roll about x
    q[3:7] = [math.cos(th / 2), math.sin(th / 2), 0, 0]
    obs = S.observe(spec, q, v, None)
    np.testing.assert_allclose(obs[0:3], [0, -math.sin(th), -math.cos(th)], atol=1e-14)
    q[3:7] = [math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)]        # yaw 90 deg
    v[0:3] = [1.0, 0.0, 0.0]
    v[3:6] = [0.1, 0.2, 0.3]
    obs = S.observe(spec, q, v, np.arange(spec.nu, dtype=float))
    np.testing.assert_allclose(obs[3:6], [0, -1, 0], atol=1e-14)         # world +x seen from a base facing +y
    np.testing.assert_allclose(obs[6:9], [0.1, 0.2, 0.3])
    nh = spec.njnt - 1
    assert obs.shape == (9 + 2 * nh + spec.nu,)
    np.testing.assert_allclose(obs[9:9 + nh], 0.0)                        # reset pose
    np.testing.assert_allclose(obs[9 + 2 * nh:], np.arange(spec.nu))


def test_resting_box_force_on_box_and_world():
    mass = 2.0
    spec = I.free_body(I.BOX, (0.1, 0.1, 0.05), mass=mass, pos=(0, 0, 0.05))
    o = Oracle(spec)
    q, v, a = spec.qpos_reset.copy(), np.zeros(6), np.zeros(6)
    for _ in range(300):
        r = o.step(q, v, a, None, want_contacts=True)
        q, v, a = r["qpos"], r["qvel"], r["qacc"]
    f_box = S.body_force(r["contacts"], 1)
    np.testing.assert_allclose(f_box, [0, 0, mass * 9.81], atol=1e-8)
    np.testing.assert_allclose(S.body_force(r["contacts"], 0), -f_box)


def test_air_time_bookkeeping_by_hand():
    dt, thr = 0.02, 1.0
    seq = [0.0, 0.0, 0.0, 5.0, 5.0, 0.5, 0.0, 9.0]
    s = np.zeros(4)
    out = []
    for fz in seq:
        s = S.air_time_update(s, np.array([0.0, 0.0, fz]), thr, dt)
        out.append(s.copy())
    # three air steps, touchdown (last air time 0.06), contact 0.04, lift-off, two air, touchdown
    np.testing.assert_allclose(out[2], [0, 0.06, 0, 0])
    np.testing.assert_allclose(out[3], [1, 0, 0.02, 0.06])
    np.testing.assert_allclose(out[4], [1, 0, 0.04, 0.06])
    np.testing.assert_allclose(out[5], [0, 0.02, 0, 0.06])
    np.testing.assert_allclose(out[7], [1, 0, 0.02, 0.04])
