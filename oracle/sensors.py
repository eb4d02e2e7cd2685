"""Observation terms and the contact sensor, FP64 (TEST INFRASTRUCTURE ONLY).

Plain numpy restatements of what the GPU readouts compute, from their definitions:
  * the velocity task's observation terms (section "Manager-Based API", Observe): the
    gravity direction and the base linear velocity expressed in the base frame (the
    transpose of the base rotation applied to world vectors), the base angular velocity
    (already body-frame in the qvel convention), joint positions relative to the reset
    pose, joint velocities, the last targets;
  * the contact sensor (section "Components"): the net force on a body summed over the
    contacts it is part of (+F on body 2, -F on body 1 of a contact), and the air-time
    bookkeeping: touchdown when |F| exceeds a threshold ends the air phase (its duration
    becomes the last air time), lift-off ends the contact phase.
"""
from __future__ import annotations

import numpy as np

FREE = 0


def quat_to_matrix(q) -> np.ndarray:
    """Rotation matrix of a unit quaternion (w, x, y, z), body to world."""
    w, x, y, z = np.asarray(q, dtype=np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def observe(spec, qpos, qvel, ctrl) -> np.ndarray:
    qpos = np.asarray(qpos, dtype=np.float64)
    qvel = np.asarray(qvel, dtype=np.float64)
    qa, da = spec.jnt_qposadr(), spec.jnt_dofadr()
    head = np.zeros(9)
    if spec.njnt and spec.jnt_type[0] == FREE:
        R = quat_to_matrix(qpos[3:7])
        g = np.asarray(spec.opt.gravity, dtype=np.float64)
        g = g / np.linalg.norm(g) if np.linalg.norm(g) > 0 else np.array([0.0, 0.0, -1.0])
        head[0:3] = R.T @ g
        head[3:6] = R.T @ qvel[0:3]
        head[6:9] = qvel[3:6]
    hs = [j for j in range(spec.njnt) if spec.jnt_type[j] != FREE]
    qrel = np.array([qpos[qa[j]] - spec.qpos_reset[qa[j]] for j in hs])
    qd = np.array([qvel[da[j]] for j in hs])
    u = np.zeros(spec.nu) if ctrl is None else np.asarray(ctrl, dtype=np.float64)
    return np.concatenate([head, qrel, qd, u])


def body_force(contacts, body) -> np.ndarray:
    """Net world-frame force on `body` from contact records (rows of the oracle's
    24-column layout: b1 at 2, b2 at 3, world force at 21..23)."""
    f = np.zeros(3)
    for c in contacts:
        if int(c[3]) == body:
            f += c[21:24]
        elif int(c[2]) == body:
            f -= c[21:24]
    return f


def air_time_update(state, force, threshold, dt) -> np.ndarray:
    """One step of the (in contact, air time, contact time, last air time) state."""
    s = np.array(state, dtype=np.float64)
    touch = np.linalg.norm(force) > threshold
    if touch:
        if s[0] < 0.5:
            s[3] = s[1]
            s[1] = 0.0
        s[2] += dt
    else:
        if s[0] > 0.5:
            s[2] = 0.0
        s[1] += dt
    s[0] = 1.0 if touch else 0.0
    return s
