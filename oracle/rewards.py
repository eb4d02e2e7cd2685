"""Reward terms, stop conditions and the contact-force history, FP64 (TEST INFRASTRUCTURE
ONLY).

Plain numpy restatements, from their definitions, of what the GPU's fused reward
launch and force-history ring compute; they share nothing with the CUDA path:
  * the reward manager of section "Manager-Based API": a weighted sum of per-world terms,
    each scaled by the control timestep, with per-term episodic sums and per-term
    detection of non-finite values (left out of the sum and reported);
  * the velocity-tracking terms of section "Tasks": tracking of a commanded planar
    velocity and yaw rate (Gaussian kernels), penalties on vertical velocity, roll/pitch
    rates, action rate, joint-limit violation, foot slip and joint accelerations, a feet
    air-time bonus at touchdown, and the tilt of the gravity direction in the base frame;
  * the termination manager's conditions: non-finite state, base below a height, base
    tilted beyond an angle, contact of an illegal body, time-out;
  * the contact sensor's force history (section "Components"): a ring of the last depth
    env steps' forces, slot (step count - 1) mod depth.
Foot velocities come from the oracle's dense point Jacobian (orc_body_jacobian), base
quantities from the free joint's quaternion.
"""
from __future__ import annotations

import math

import numpy as np

from .sensors import FREE, quat_to_matrix

TERMS = ("track_lin_vel", "track_ang_vel", "lin_vel_z", "ang_vel_xy", "action_rate", "joint_limit",
         "feet_slip", "feet_air_time", "upright", "joint_acc")
TERMINATED, TIMEOUT, NONFINITE, LOW, TILT, ILLEGAL = 1, 2, 4, 8, 16, 32


def raw_terms(oracle, spec, qpos, qvel, qacc, cmd, action, prev_action, sensor_state, feet, cfg) -> np.ndarray:
    """The ten raw term values of one world (FP64)."""
    qpos, qvel, qacc = (np.asarray(x, dtype=np.float64) for x in (qpos, qvel, qacc))
    raw = np.zeros(len(TERMS))
    if spec.njnt and spec.jnt_type[0] == FREE:
        R = quat_to_matrix(qpos[3:7])                 # base -> world
        g = np.asarray(spec.opt.gravity, dtype=np.float64)
        g = g / np.linalg.norm(g) if np.linalg.norm(g) > 0 else np.array([0.0, 0.0, -1.0])
        vb = R.T @ qvel[0:3]                           # base-frame linear velocity
        wb = qvel[3:6]                                 # the free joint's angular velocity is body-frame
        gb = R.T @ g
        raw[0] = math.exp(-((vb[0] - cmd[0]) ** 2 + (vb[1] - cmd[1]) ** 2) / cfg["sigma_lin"] ** 2)
        raw[1] = math.exp(-((wb[2] - cmd[2]) ** 2) / cfg["sigma_ang"] ** 2)
        raw[2] = vb[2] ** 2
        raw[3] = wb[0] ** 2 + wb[1] ** 2
        raw[8] = gb[0] ** 2 + gb[1] ** 2
    if spec.nu and action is not None:
        raw[4] = float(np.sum((np.asarray(action, dtype=np.float64) - np.asarray(prev_action, dtype=np.float64)) ** 2))
    if getattr(spec, "jnt_limited", None) is not None:
        qa = spec.jnt_qposadr()
        for j in range(spec.njnt):
            if spec.jnt_limited[j]:
                lo, hi = spec.jnt_range[j]
                q = qpos[qa[j]]
                raw[5] += max(0.0, lo - q) + max(0.0, q - hi)
    if len(feet):
        f = oracle.fk(qpos)
        for k, b in enumerate(feet):
            Jp, _ = oracle.body_jacobian(qpos, int(b), f["xpos"][b])
            v = Jp @ qvel
            st = sensor_state[k]
            if st[0] > 0.5:
                raw[6] += v[0] ** 2 + v[1] ** 2
                if st[2] <= 1.5 * cfg["dt"]:
                    raw[7] += st[3] - cfg["air_time_target"]
    da = spec.jnt_dofadr()
    for j in range(spec.njnt):
        if spec.jnt_type[j] != FREE:
            raw[9] += qacc[da[j]] ** 2
    return raw


def reward(oracle, spec, qpos, qvel, qacc, cmd, action, prev_action, sensor_state, feet, cfg, contacts=None,
           illegal=(), step_count=0, nan_status=False):
    """(reward, per-term contributions weight x raw x dt, done bits) of one world."""
    raw = raw_terms(oracle, spec, qpos, qvel, qacc, cmd, action, prev_action, sensor_state, feet, cfg)
    w = np.asarray(cfg["weight"], dtype=np.float64)
    contrib = np.where(w != 0.0, w * raw * cfg["dt"], 0.0)
    done = 0
    for k in range(len(TERMS)):
        if not np.isfinite(contrib[k]):
            done |= 256 << k
            contrib[k] = 0.0
    state_bad = nan_status or not (np.all(np.isfinite(qpos)) and np.all(np.isfinite(qvel))
                                   and np.all(np.isfinite(qacc)))
    if state_bad:
        done |= NONFINITE
    if spec.njnt and spec.jnt_type[0] == FREE:
        if cfg["min_base_height"] > 0 and qpos[2] < cfg["min_base_height"]:
            done |= LOW
        if cfg["max_tilt"] > 0:
            R = quat_to_matrix(qpos[3:7])
            up = R[:, 2]                               # base up axis in the world
            g = np.asarray(spec.opt.gravity, dtype=np.float64)
            gu = -g / np.linalg.norm(g) if np.linalg.norm(g) > 0 else np.array([0.0, 0.0, 1.0])
            if float(up @ gu) < math.cos(cfg["max_tilt"]):
                done |= TILT
    if len(illegal) and contacts is not None:
        ill = set(int(b) for b in illegal)
        if any(int(c[2]) in ill or int(c[3]) in ill for c in contacts):
            done |= ILLEGAL
    if done & (NONFINITE | LOW | TILT | ILLEGAL):
        done |= TERMINATED
    if cfg["max_episode_steps"] > 0 and step_count >= cfg["max_episode_steps"]:
        done |= TIMEOUT
    return float(np.sum(contrib)), contrib, done


def history_write(ring: np.ndarray, step_count: int, force) -> None:
    """Write one env step's force into a [depth, 3] ring (slot (step count - 1) mod depth)."""
    depth = ring.shape[0]
    ring[(step_count - 1) % depth] = force


def history_oldest_first(ring: np.ndarray, step_count: int) -> np.ndarray:
    """The ring's forces oldest first (the last min(step count, depth) env steps)."""
    depth = ring.shape[0]
    n = min(step_count, depth)
    return np.array([ring[(step_count - n + i) % depth] for i in range(n)]).reshape(n, 3)
