"""Pins of the oracle's reward terms, stop conditions and force-history ring (CPU):
closed forms for a world at rest and for known velocities, an independent rotation
(scipy) for base-frame quantities, a free body whose foot velocity is its own, a
hand-worked touchdown, and the ring read back in order."""
import math

import numpy as np
from scipy.spatial.transform import Rotation

from oracle import Oracle
from oracle import rewards as RW
from paper_2601_22074_b300 import inputs as I

CFG = dict(weight=[1.0, 0.5, -2.0, -0.05, -0.01, -10.0, -0.1, 1.0, -1.0, -2.5e-7], sigma_lin=0.5, sigma_ang=0.5,
           air_time_target=0.4, dt=0.02, min_base_height=0.3, max_tilt=1.0, max_episode_steps=1000)


def _rest(spec):
    o = Oracle(spec)
    q = np.array(spec.qpos_reset, dtype=np.float64)
    return o, q, np.zeros(spec.nv), np.zeros(spec.nv)


def test_world_at_rest_with_zero_command_earns_the_tracking_weights():
    spec = I.quadruped()
    o, q, v, a = _rest(spec)
    act = spec.qpos_reset[spec.act_qposadr()]
    r, c, done = RW.reward(o, spec, q, v, a, np.zeros(3), act, act, np.zeros((0, 4)), [], CFG)
    assert abs(r - (1.0 + 0.5) * 0.02) < 1e-15 and done == 0
    assert np.allclose(c[2:], 0.0)


def test_base_frame_velocity_and_tilt_match_an_independent_rotation():
    spec = I.quadruped()
    o, q, v, a = _rest(spec)
    rot = Rotation.from_euler("zyx", [0.7, 0.2, -0.3])
    x, y, z, w = rot.as_quat()
    q[3:7] = [w, x, y, z]
    v[0:3] = [0.8, -0.4, 0.3]
    v[3:6] = [0.1, -0.2, 0.6]
    cmd = np.array([0.5, 0.2, 0.4])
    raw = RW.raw_terms(o, spec, q, v, a, cmd, None, None, np.zeros((0, 4)), [], CFG)
    vb = rot.inv().apply(v[0:3])
    gb = rot.inv().apply([0.0, 0.0, -1.0])
    assert abs(raw[0] - math.exp(-((vb[0] - 0.5) ** 2 + (vb[1] - 0.2) ** 2) / 0.25)) < 1e-12
    assert abs(raw[1] - math.exp(-(0.6 - 0.4) ** 2 / 0.25)) < 1e-12
    assert abs(raw[2] - vb[2] ** 2) < 1e-12 and abs(raw[3] - 0.05) < 1e-12
    assert abs(raw[8] - (gb[0] ** 2 + gb[1] ** 2)) < 1e-12
    tilt = math.acos(rot.apply([0.0, 0.0, 1.0])[2])
    cfg = dict(CFG, max_tilt=tilt * 0.99, min_base_height=0.0)
    assert RW.reward(o, spec, q, v, a, cmd, None, None, np.zeros((0, 4)), [], cfg)[2] == RW.TILT | RW.TERMINATED
    cfg = dict(CFG, max_tilt=tilt * 1.01, min_base_height=0.0)
    assert RW.reward(o, spec, q, v, a, cmd, None, None, np.zeros((0, 4)), [], cfg)[2] == 0


def test_foot_slip_of_a_free_body_is_its_planar_speed_squared():
    spec = I.free_body(I.SPHERE, (0.1,), pos=(0, 0, 0.5))
    o = Oracle(spec)
    q = np.array(spec.qpos_reset, dtype=np.float64)
    v = np.array([0.3, -0.4, 2.0, 0.0, 0.0, 0.0])
    st = np.array([[1.0, 0.0, 0.5, 0.3]])        # in contact for 0.5 s: no touchdown
    raw = RW.raw_terms(o, spec, q, v, np.zeros(6), np.zeros(3), None, None, st, [1], CFG)
    assert abs(raw[6] - 0.25) < 1e-12 and raw[7] == 0.0
    v[3:6] = [0.0, 0.0, 1.5]                      # spin about the origin's own z: no slip added
    assert abs(RW.raw_terms(o, spec, q, v, np.zeros(6), np.zeros(3), None, None, st, [1], CFG)[6] - 0.25) < 1e-12


def test_air_time_bonus_only_at_touchdown():
    spec = I.free_body(I.SPHERE, (0.1,), pos=(0, 0, 0.5))
    o = Oracle(spec)
    q = np.array(spec.qpos_reset, dtype=np.float64)
    z = np.zeros(6)
    td = np.array([[1.0, 0.0, 0.02, 0.55]])      # touched down this step after 0.55 s in the air
    assert abs(RW.raw_terms(o, spec, q, z, z, np.zeros(3), None, None, td, [1], CFG)[7] - 0.15) < 1e-12
    later = np.array([[1.0, 0.0, 0.04, 0.55]])
    assert RW.raw_terms(o, spec, q, z, z, np.zeros(3), None, None, later, [1], CFG)[7] == 0.0


def test_stop_conditions_and_nonfinite_terms():
    spec = I.quadruped()
    o, q, v, a = _rest(spec)
    q[2] = 0.2
    con = np.zeros((1, 24))
    con[0, 2:4] = [0, 1]                          # the base (body 1) touches the floor
    _, _, done = RW.reward(o, spec, q, v, a, np.zeros(3), None, None, np.zeros((0, 4)), [], CFG, contacts=con,
                           illegal=[1], step_count=1000)
    assert done == RW.TERMINATED | RW.LOW | RW.ILLEGAL | RW.TIMEOUT
    act = np.zeros(spec.nu)
    bad = act.copy()
    bad[3] = np.nan
    r, c, done = RW.reward(o, spec, q, v, a, np.zeros(3), bad, act, np.zeros((0, 4)), [], dict(CFG, min_base_height=0))
    assert done == 256 << 4 and np.isfinite(r) and c[4] == 0.0
    v[0] = np.inf
    assert RW.reward(o, spec, q, v, a, np.zeros(3), act, act, np.zeros((0, 4)), [],
                     dict(CFG, min_base_height=0))[2] & (RW.NONFINITE | RW.TERMINATED) == RW.NONFINITE | RW.TERMINATED


def test_joint_limit_violation_sums_distances_outside_the_range():
    spec = I.with_limits(I.quadruped(), 0.3)
    o, q, v, a = _rest(spec)
    qa = spec.jnt_qposadr()
    q[qa[1]] += 0.5                               # 0.2 above its upper limit
    q[qa[2]] -= 0.45                              # 0.15 below its lower limit
    assert abs(RW.raw_terms(o, spec, q, v, a, np.zeros(3), None, None, np.zeros((0, 4)), [], CFG)[5] - 0.35) < 1e-12


def test_force_history_ring_reads_back_oldest_first():
    ring = np.zeros((3, 3))
    forces = [np.full(3, float(k)) for k in range(1, 6)]
    for s, f in enumerate(forces, start=1):
        RW.history_write(ring, s, f)
    assert np.array_equal(RW.history_oldest_first(ring, 5), np.array(forces[2:]))
    assert np.array_equal(RW.history_oldest_first(np.zeros((3, 3)), 0), np.zeros((0, 3)))
