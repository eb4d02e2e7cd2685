"""Differential inverse kinematics by damped least squares, FP64 (TEST INFRASTRUCTURE ONLY).

The action term of the paper's manager-based API (section "Manager-Based API", action
manager: differential IK): for a point fixed to a body, with the Jacobian J restricted to
the actuated joints' columns, the joint update minimising |J dq - e|^2 + lambda^2 |dq|^2,
    dq = J^T (J J^T + lambda^2 I)^-1 e,
e = (target position - position) and, when a target orientation is given, the rotation
vector of q_target (x) q^-1 (world frame). The targets handed to the PD servos are the
actuated joints' positions plus dq.
"""
from __future__ import annotations

import numpy as np

from .sensors import quat_to_matrix


def quat_mul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def rotation_vector(q) -> np.ndarray:
    """Axis times angle of the unit quaternion q (w, x, y, z), angle in [0, pi]."""
    q = np.asarray(q, dtype=np.float64)
    if q[0] < 0:
        q = -q
    s = np.linalg.norm(q[1:])
    if s == 0:
        return np.zeros(3)
    return 2.0 * np.arctan2(s, q[0]) * q[1:] / s


def diffik(o, spec, qpos, body, offset, target_pos, target_quat=None, lam=0.05):
    """Returns (ctrl targets [nu], dq [nu], error vector e)."""
    f = o.fk(qpos)
    R = f["xmat"][body]
    p = f["xpos"][body] + R @ np.asarray(offset, dtype=np.float64)
    Jp, Jr = o.body_jacobian(qpos, body, p)
    cols = [spec.jnt_dofadr()[j] for j in spec.act_jnt]
    e = np.asarray(target_pos, dtype=np.float64) - p
    J = Jp[:, cols]
    if target_quat is not None:
        qc = f["xquat"][body]
        qerr = quat_mul(np.asarray(target_quat, dtype=np.float64), qc * np.array([1, -1, -1, -1]))
        e = np.concatenate([e, rotation_vector(qerr)])
        J = np.vstack([J, Jr[:, cols]])
    y = np.linalg.solve(J @ J.T + lam * lam * np.eye(J.shape[0]), e)
    dq = J.T @ y
    qa = [spec.jnt_qposadr()[j] for j in spec.act_jnt]
    return np.asarray(qpos, dtype=np.float64)[qa] + dq, dq, e
