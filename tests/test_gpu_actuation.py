"""Joint limits, DC-motor saturation and actuation delay on the GPU (section
"Components": actuators with velocity-dependent saturation and delay; MuJoCo's joint
limits as constraint rows), against the FP64 oracle where the oracle models them."""
import numpy as np
import pytest
import torch

from paper_2601_22074_b300 import build, inputs as I
from paper_2601_22074_b300.batch import Batch, Model

pytestmark = pytest.mark.gpu
TOL_CONTACT = 1e-3
PLACEMENTS = [pytest.param({}, id="fused"), pytest.param(dict(working_set=2, warps_per_block=2), id="staged"),
              pytest.param(dict(working_set=3, warps_per_block=4, schedule=1), id="grouped")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _check(rep, tol=TOL_CONTACT):
    from parity import check
    print("limit steps", rep.limit_steps)
    check(rep, tol)


@pytest.mark.parametrize("options", PLACEMENTS)
def test_humanoid_with_joint_limits_matches_oracle(options):
    """Every hinge limited to its reset angle +- 0.3 rad; the N(0, 0.3) targets drive many
    joints into their limits, so limit rows are active alongside the foot contacts."""
    from parity import teacher_forced
    spec = I.with_limits(I.humanoid(), 0.3)
    rep = teacher_forced(spec, W=48, nsteps=12, decimation=4, warm_steps=40, options=options)
    assert rep.limit_steps > 100 and rep.contact_steps > 100
    _check(rep)


@pytest.mark.parametrize("options", PLACEMENTS)
def test_pendulum_limits_without_contacts_match_oracle(options):
    """Limit rows alone (no collision pairs): a 3-link pendulum with +-0.5 rad ranges, reset
    angles up to +-1.2 rad (most worlds start beyond a limit and are pushed back)."""
    from parity import teacher_forced
    spec = I.with_limits(I.pendulum(3, noise=1.2), 0.5)
    rep = teacher_forced(spec, W=64, nsteps=60, decimation=1, contacts=False, options=options)
    assert rep.limit_steps > 200
    _check(rep)


@pytest.mark.parametrize("options", PLACEMENTS)
def test_quadruped_with_dc_motors_matches_oracle(options):
    """Stall torque 15 N m, no-load speed 20 rad/s, limit 8 N m on every leg joint: the
    kp = 40 servo saturates on most steps."""
    from parity import teacher_forced
    spec = I.with_dcmotor(I.quadruped(), 15.0, 20.0, 8.0)
    rep = teacher_forced(spec, W=48, nsteps=20, decimation=4, warm_steps=20, options=options)
    assert rep.contact_steps > 100
    _check(rep)


@pytest.mark.parametrize("options", PLACEMENTS)
def test_actuation_delay_is_a_shift_of_the_targets(options):
    """With a delay of D env steps the step equals the undelayed step fed the targets of
    D steps earlier (the reset pose for the first D steps), bitwise; the delayed targets
    survive a checkpoint round trip."""
    D, W, T = 3, 64, 12
    base = I.quadruped()
    spec_d = I.with_delay(base, D)
    ctrl = I.ctrl_targets(base, W, T, 5).astype(np.float32)
    hold = np.tile(base.qpos_reset[base.act_qposadr()].astype(np.float32), (W, 1))
    shifted = np.concatenate([np.repeat(hold[None], D, axis=0), ctrl[:-D]], axis=0)
    a = Batch(Model(spec_d), W, **options)
    b = Batch(Model(base), W, **options)
    a.reset(4)
    b.reset(4)
    ca = torch.tensor(ctrl, device="cuda")
    cb = torch.tensor(shifted, device="cuda")
    snap = None
    for t in range(T):
        a.step(ca[t].reshape(-1), 4)
        b.step(cb[t].reshape(-1), 4)
        if t == 5:
            snap = a.state_save()
    torch.cuda.synchronize()
    for f in ("qpos", "qvel", "qacc"):
        assert torch.equal(a.get(f), b.get(f)), f
    end = a.get("qpos").clone()
    a.state_restore(snap)
    for t in range(6, T):
        a.step(ca[t].reshape(-1), 4)
    torch.cuda.synchronize()
    assert torch.equal(a.get("qpos"), end)


@pytest.mark.parametrize("options", PLACEMENTS)
def test_actuation_delay_matches_oracle_delay_model(options):
    """Delay of D = 3 env steps, teacher-forced from the reset: the oracle applies the
    reset pose for s < D and the target submitted at s - D after (its own model of the
    delay), the GPU keeps the submitted targets in its per-world history."""
    from oracle.actuation import delayed_targets
    from parity import teacher_forced
    D = 3
    spec = I.with_delay(I.quadruped(), D)
    rep = teacher_forced(spec, W=32, nsteps=10, decimation=4, options=options,
                         oracle_ctrl_fn=lambda c: delayed_targets(spec, c, D))
    assert rep.compared >= 0.98 * 32 * 10
    _check(rep)


@pytest.mark.parametrize("options", PLACEMENTS)
def test_quadruped_with_randomised_body_inertias_matches_oracle(options):
    """Per-world masses, centres of mass and inertias drawn in log-Cholesky coordinates
    (sigma 0.05) and set through the body-inertia parameter."""
    from parity import teacher_forced
    rep = teacher_forced(I.quadruped(), W=48, nsteps=15, decimation=4, warm_steps=20, options=options,
                         inertia_sigma=0.05)
    assert rep.contact_steps > 100
    _check(rep)
