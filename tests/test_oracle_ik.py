"""Pins of the oracle's body Jacobians and damped-least-squares IK (CPU): central finite
differences of forward kinematics, the normal equations of the damped least-squares
problem, and convergence to a reachable target."""
import numpy as np

from oracle import Oracle
from oracle import ik as IK
from paper_2601_22074_b300 import inputs as I
from test_oracle_pins import advance_qpos, random_state


def _point(o, q, body, off):
    f = o.fk(q)
    return f["xpos"][body] + f["xmat"][body] @ off, f["xmat"][body]


def test_body_jacobians_match_finite_differences():
    rng = np.random.default_rng(3)
    for spec, body in ((I.manipulation(), 7), (I.humanoid(), 23), (I.humanoid(), 30), (I.quadruped(), 4)):
        o = Oracle(spec)
        for _ in range(3):
            q, _ = random_state(spec, rng)
            off = rng.normal(0, 0.05, 3)
            p, _ = _point(o, q, body, off)
            Jp, Jr = o.body_jacobian(q, body, p)
            eps = 1e-6
            for d in range(spec.nv):
                e = np.zeros(spec.nv)
                e[d] = 1.0
                pp, Rp = _point(o, advance_qpos(spec, q, e, eps), body, off)
                pm, Rm = _point(o, advance_qpos(spec, q, e, -eps), body, off)
                np.testing.assert_allclose(Jp[:, d], (pp - pm) / (2 * eps), atol=1e-7)
                Om = ((Rp - Rm) / (2 * eps)) @ _point(o, q, body, off)[1].T
                np.testing.assert_allclose(Jr[:, d], [Om[2, 1], Om[0, 2], Om[1, 0]], atol=1e-7)


def test_dls_step_solves_the_normal_equations():
    rng = np.random.default_rng(4)
    spec = I.manipulation()
    o = Oracle(spec)
    for lam in (0.01, 0.1, 1.0):
        q, _ = random_state(spec, rng, qscale=0.3)
        tp = rng.normal(0, 0.1, 3) + o.fk(q)["xpos"][7]
        tq = rng.normal(size=4)
        tq /= np.linalg.norm(tq)
        for quat in (None, tq):
            ctrl, dq, e = IK.diffik(o, spec, q, 7, [0, 0, 0.05], tp, quat, lam)
            f = o.fk(q)
            p = f["xpos"][7] + f["xmat"][7] @ np.array([0, 0, 0.05])
            Jp, Jr = o.body_jacobian(q, 7, p)
            cols = [spec.jnt_dofadr()[j] for j in spec.act_jnt]
            J = Jp[:, cols] if quat is None else np.vstack([Jp[:, cols], Jr[:, cols]])
            np.testing.assert_allclose(J.T @ (J @ dq - e) + lam * lam * dq, 0.0, atol=1e-10)


def test_iterated_dls_reaches_a_reachable_pose():
    """Target = the pose of the end-effector point at another configuration; repeated DLS
    steps on the actuated joints (no dynamics) bring position and orientation there."""
    spec = I.manipulation()
    o = Oracle(spec)
    rng = np.random.default_rng(5)
    qa = [spec.jnt_qposadr()[j] for j in spec.act_jnt]
    off = np.array([0.0, 0.0, 0.05])
    for _ in range(3):
        q = spec.qpos_reset.copy()
        qt = q.copy()
        qt[qa[:7]] += rng.uniform(-0.4, 0.4, 7)
        ft = o.fk(qt)
        tp = ft["xpos"][7] + ft["xmat"][7] @ off
        tq = ft["xquat"][7]
        for it in range(60):
            ctrl, dq, e = IK.diffik(o, spec, q, 7, off, tp, tq, 0.05)
            q[qa] = ctrl
        assert np.linalg.norm(e) < 1e-6, np.linalg.norm(e)
