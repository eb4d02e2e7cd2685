"""Damped-least-squares differential IK on the GPU against the oracle's (oracle/ik.py)
on the same states; and closed-loop reaching through the physics step."""
import numpy as np
import pytest
import torch

from paper_2601_22074_b300 import build, inputs as I
from paper_2601_22074_b300.batch import Batch, Model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


@pytest.mark.parametrize("with_quat", [False, True])
def test_diffik_matches_oracle(with_quat):
    from oracle import Oracle, ik as IK
    spec = I.manipulation()
    other = I.quadruped()
    W, Wq = 32, 16
    b = Batch([Model(other), Model(spec)], [Wq, W])
    b.reset(3)
    ctrl_m = torch.tensor(I.ctrl_targets(spec, W, 10, 4), dtype=torch.float32, device="cuda")
    ctrl_q = torch.tensor(I.ctrl_targets(other, Wq, 10, 4), dtype=torch.float32, device="cuda")
    for t in range(10):
        b.step(torch.cat([ctrl_q[t].reshape(-1), ctrl_m[t].reshape(-1)]), 4)
    o = Oracle(spec)
    q = b.group_view(b.get("qpos"), "qpos", 1).double().cpu().numpy()
    rng = np.random.default_rng(7)
    off = [0.0, 0.0, 0.05]
    tp, tq = [], []
    for w in range(W):
        f = o.fk(q[w])
        tp.append(f["xpos"][7] + rng.normal(0, 0.05, 3))
        qq = f["xquat"][7] + rng.normal(0, 0.1, 4)
        tq.append(qq / np.linalg.norm(qq))
    tp, tq = np.array(tp), np.array(tq)
    flat = torch.full((Wq * other.nu + W * spec.nu,), 7.0, dtype=torch.float32, device="cuda")
    b.diffik(1, 7, off, torch.tensor(tp), flat, torch.tensor(tq) if with_quat else None, damping=0.05)
    torch.cuda.synchronize()
    out = flat.double().cpu().numpy()
    assert np.all(out[: Wq * other.nu] == 7.0)              # the other group is untouched
    got = out[Wq * other.nu:].reshape(W, spec.nu)
    for w in range(W):
        want, dq, e = IK.diffik(o, spec, q[w], 7, off, tp[w], tq[w] if with_quat else None, 0.05)
        qa = q[w][[spec.jnt_qposadr()[j] for j in spec.act_jnt]]
        err = np.abs(got[w] - want).max() / max(np.abs(dq).max(), 1e-3)
        assert err < 2e-3, (w, err, got[w] - qa, dq)


def test_diffik_closed_loop_reaches_a_target_through_the_physics():
    """Each env step: IK targets toward a fixed reachable point, then a physics step; the
    end-effector point settles near the target, within the offset a PD servo leaves under
    gravity (kp 500: a few centimetres at most), from a start about 15 cm away."""
    from oracle import Oracle
    spec = I.manipulation(arm_kp=500.0, arm_kd=1.0)
    W = 16
    b = Batch(Model(spec), W)
    b.reset(1)
    o = Oracle(spec)
    q0 = spec.qpos_reset.copy()
    qa = [spec.jnt_qposadr()[j] for j in spec.act_jnt]
    q1 = q0.copy()
    q1[qa[:7]] += np.array([0.2, -0.2, 0.1, 0.2, 0.0, -0.1, 0.1])
    f1 = o.fk(q1)
    off = np.array([0.0, 0.0, 0.05])
    target = f1["xpos"][7] + f1["xmat"][7] @ off
    f0 = o.fk(q0)
    d0 = np.linalg.norm(f0["xpos"][7] + f0["xmat"][7] @ off - target)
    tp = torch.tensor(np.tile(target, (W, 1)), dtype=torch.float32, device="cuda")
    ctrl = torch.zeros(W * spec.nu, dtype=torch.float32, device="cuda")
    for t in range(150):
        b.diffik(0, 7, off, tp, ctrl, damping=0.05)
        b.step(ctrl, 4)
    q = b.get("qpos").view(W, spec.nq).double().cpu().numpy()
    for w in range(W):
        f = o.fk(q[w])
        p = f["xpos"][7] + f["xmat"][7] @ off
        assert np.linalg.norm(p - target) < min(0.03, 0.25 * d0), (w, np.linalg.norm(p - target), d0)
