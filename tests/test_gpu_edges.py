"""Edge cases of the step on the GPU: ragged and tiny world counts in every placement,
empty groups, contact overflow beyond the model's cap, and closed-form degenerate motions
(free fall, torque-free spin)."""
import math

import numpy as np
import pytest
import torch

from paper_2601_22074_b300 import _lib as L, build, inputs as I
from paper_2601_22074_b300.batch import Batch, Model

pytestmark = pytest.mark.gpu
PLACEMENTS = [pytest.param({}, id="fused"), pytest.param(dict(working_set=2, warps_per_block=2), id="staged"),
              pytest.param(dict(working_set=3, warps_per_block=4, schedule=1), id="grouped"),
              pytest.param(dict(working_set=3, warps_per_block=4, schedule=1, lane_solve=1), id="lane")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


@pytest.mark.parametrize("options", PLACEMENTS)
@pytest.mark.parametrize("W", [1, 3, 37])
def test_ragged_world_counts_match_oracle(W, options):
    """World counts that fill no CTA or leave a ragged last one (4 worlds per CTA, 32 per
    lane warp): every world still matches the oracle."""
    from parity import check, teacher_forced
    rep = teacher_forced(I.quadruped(), W=W, nsteps=4, decimation=4, warm_steps=20, options=options)
    assert rep.compared + rep.mismatches == 4 * W
    check(rep, 1e-3, max_mismatch=0.1)


@pytest.mark.parametrize("options", PLACEMENTS[:3])
def test_empty_groups_step_and_leave_the_others_unchanged(options):
    """A batch whose first and last groups hold no worlds steps like the batch without them
    (bitwise), and a batch with no worlds at all steps as a no-op."""
    spec = I.quadruped()
    W = 24
    ctrl = torch.tensor(I.ctrl_targets(spec, W, 5, 2), dtype=torch.float32, device="cuda").reshape(5, -1)
    a = Batch([Model(I.pendulum(3)), Model(spec), Model(I.humanoid())], [0, W, 0], **options)
    b = Batch(Model(spec), W, **options)
    for x in (a, b):
        x.reset(9)
        for t in range(5):
            x.step(ctrl[t], 4)
    torch.cuda.synchronize()
    for f in ("qpos", "qvel", "qacc"):
        assert torch.equal(a.get(f), b.get(f)), f
    e = Batch(Model(spec), 0, **options)
    e.reset(1)
    e.step(torch.zeros(1, device="cuda"), 4)
    torch.cuda.synchronize()
    assert e.get("qpos").numel() == 0


@pytest.mark.parametrize("options", PLACEMENTS[:3])
def test_contact_overflow_is_flagged_and_matches_the_capped_oracle(options):
    """With the model's contact cap at 2 the quadruped often has more touching feet: those
    worlds carry the overflow bit, keep the first two contacts in pair order, and still
    match the oracle, which applies the same cap."""
    from parity import check, teacher_forced
    spec = I.quadruped(contact_cap=2)
    assert Model(spec).ncon_max == 2
    rep = teacher_forced(spec, W=32, nsteps=6, decimation=4, warm_steps=20, options=options)
    check(rep, 1e-3)
    b = Batch(Model(spec), 32, **options)
    b.reset(0)
    ctrl = torch.tensor(I.ctrl_targets(spec, 32, 20, 11), dtype=torch.float32, device="cuda")
    for t in range(20):
        b.step(ctrl[t].reshape(-1), 4)
    st = b.get("status").cpu().numpy()
    assert np.any(st & L.STATUS_OVERFLOW)
    assert np.all(b.get("stats").view(32, 4).cpu().numpy()[:, 0] <= 2)


@pytest.mark.parametrize("options", PLACEMENTS[:3])
def test_free_fall_follows_the_discrete_closed_form(options):
    """A free sphere far above the ground, no contact, no actuation: semi-implicit Euler
    gives z_n = z_0 - g h^2 n (n + 1) / 2 and v_n = -g n h exactly in exact arithmetic; the
    FP32 step stays within rounding of it over 100 substeps."""
    spec = I.free_body(I.SPHERE, (0.1,), pos=(0, 0, 5.0))
    b = Batch(Model(spec), 8, **options)
    b.reset(0)
    h, g, n = spec.opt.timestep, 9.81, 25
    for _ in range(n):
        b.step(None, 4)
    torch.cuda.synchronize()
    q = b.get("qpos").view(8, spec.nq).double().cpu().numpy()
    v = b.get("qvel").view(8, spec.nv).double().cpu().numpy()
    N = 4 * n
    np.testing.assert_allclose(q[:, 2], 5.0 - g * h * h * N * (N + 1) / 2, atol=5e-5)
    np.testing.assert_allclose(v[:, 2], -g * N * h, rtol=1e-5)
    np.testing.assert_allclose(q[:, 3:7], np.tile([1, 0, 0, 0], (8, 1)), atol=1e-7)


@pytest.mark.parametrize("options", PLACEMENTS[:3])
def test_torque_free_symmetric_spin_keeps_its_rate(options):
    """Zero gravity, a symmetric body spinning about its symmetry axis: the body-frame
    angular velocity stays constant and the orientation turns at that rate."""
    spec = I.free_body(I.SPHERE, (0.1,), pos=(0, 0, 5.0), plane=False, gravity=(0.0, 0.0, 0.0))
    b = Batch(Model(spec), 4, **options)
    b.reset(0)
    w = 3.0
    v = torch.zeros(4, 6)
    v[:, 5] = w
    b.set("qvel", v.reshape(-1))
    n = 50
    for _ in range(n):
        b.step(None, 4)
    torch.cuda.synchronize()
    qv = b.get("qvel").view(4, 6).double().cpu().numpy()
    q = b.get("qpos").view(4, 7).double().cpu().numpy()
    np.testing.assert_allclose(qv[:, 5], w, rtol=1e-6)
    ang = w * spec.opt.timestep * 4 * n
    np.testing.assert_allclose(q[:, 3:7], np.tile([math.cos(ang / 2), 0, 0, math.sin(ang / 2)], (4, 1)),
                               atol=5e-5)


@pytest.mark.parametrize("options", [pytest.param({}, id="fused"),
                                     pytest.param(dict(working_set=3, warps_per_block=4, schedule=1,
                                                       lane_solve=1), id="lane")])
def test_batches_with_different_shared_memory_needs_coexist(options):
    """A batch of large worlds, then one of small worlds: the kernels' shared-memory limits
    are raised once and never lowered, so the first batch still steps (and equals a batch
    stepped alone)."""
    big, small = I.humanoid(), I.quadruped()
    ctrl = torch.tensor(I.ctrl_targets(big, 16, 3, 1), dtype=torch.float32, device="cuda").reshape(3, -1)
    a = Batch(Model(big), 16, **options)
    a.reset(2)
    a.step(ctrl[0], 4)
    b = Batch(Model(small), 8, **options)
    b.reset(2)
    b.step(torch.zeros(8 * small.nu, device="cuda"), 4)
    a.step(ctrl[1], 4)
    ref = Batch(Model(big), 16, **options)
    ref.reset(2)
    ref.step(ctrl[0], 4)
    ref.step(ctrl[1], 4)
    torch.cuda.synchronize()
    assert torch.equal(a.get("qpos"), ref.get("qpos"))
