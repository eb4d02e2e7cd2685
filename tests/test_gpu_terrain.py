"""Heightfield terrain on the GPU against the oracle: contact dynamics (teacher-forced
steps) and height-scan ray casts."""
import numpy as np
import pytest
import torch

from paper_2601_22074_b300 import build, inputs as I
from paper_2601_22074_b300.batch import Batch, Model

pytestmark = pytest.mark.gpu
PLACEMENTS = [pytest.param({}, id="fused"), pytest.param(dict(working_set=2, warps_per_block=2), id="staged"),
              pytest.param(dict(working_set=3, warps_per_block=4, schedule=1), id="grouped")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _check(rep, tol=1e-3):
    from parity import check
    check(rep, tol)


@pytest.mark.parametrize("options", PLACEMENTS)
@pytest.mark.parametrize("name", ["quadruped", "humanoid"])
def test_robots_on_bumpy_terrain_match_oracle(name, options):
    from parity import teacher_forced
    spec = I.with_terrain(getattr(I, name)(), amplitude=0.04, seed=1)
    rep = teacher_forced(spec, W=48, nsteps=12, decimation=4, warm_steps=30, options=options)
    assert rep.contact_steps > 100
    _check(rep)


def test_height_scan_on_terrain_matches_oracle():
    from oracle import Oracle, raycast as RC
    spec = I.with_terrain(I.quadruped(), amplitude=0.06, seed=2)
    W = 16
    b = Batch(Model(spec), W, working_set=2)
    b.reset(8)
    ctrl = torch.tensor(I.ctrl_targets(spec, W, 10, 2), dtype=torch.float32, device="cuda")
    for t in range(10):
        b.step(ctrl[t].reshape(-1), 4)
    xs = (np.arange(9) - 4) * 0.1
    o = np.array([[x, y, 0.3] for x in xs for y in xs[::2]])
    d = np.tile([0.0, 0.0, -1.0], (len(o), 1))
    d[::3] += np.array([0.2, -0.1, 0.0])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    dist = b.raycast(0, 1, torch.tensor(o), torch.tensor(d), max_dist=3.0).double().cpu().numpy()
    q = b.get("qpos").view(W, spec.nq).double().cpu().numpy()
    orc = Oracle(spec)
    for w in range(W):
        ref = RC.raycast(orc, spec, q[w], 1, o, d, 3.0, True)
        np.testing.assert_allclose(dist[w], ref, atol=3e-5, rtol=1e-5)
        assert np.all(ref < 3.0)


@pytest.mark.parametrize("options", PLACEMENTS)
def test_boxes_on_bumps_touch_the_terrain_at_convex_vertices(options):
    """Free boxes dropped onto Gaussian bumps of a 0.05 m grid: bump crests press into the
    box faces between the box's vertices (convex grid vertices inside the box), beside the
    vertex contacts; one env step at a time against the oracle, contact records compared
    one by one."""
    import dataclasses
    from parity import teacher_forced
    terrain = I.with_terrain(I.quadruped(), nrow=41, ncol=41, half=1.0, amplitude=0.12, seed=7).hfield_data
    spec0 = I.free_body(I.BOX, (0.12, 0.07, 0.04), mass=1.0, pos=(0.1, -0.2, 0.35))
    gt = spec0.geom_type.copy()
    gt[0] = I.HFIELD
    spec = dataclasses.replace(spec0, geom_type=gt, hfield_data=terrain, hfield_size=(1.0, 1.0))
    W = 32
    rng = np.random.default_rng(5)
    q0 = np.tile(spec.qpos_reset, (W, 1))
    q0[:, 0:2] = rng.uniform(-0.6, 0.6, (W, 2))
    q0[:, 2] = 0.25
    qq = rng.normal(size=(W, 4)) * np.array([4.0, 0.3, 0.3, 1.0])    # mostly yaw
    q0[:, 3:7] = qq / np.linalg.norm(qq, axis=1, keepdims=True)
    rep = teacher_forced(spec, W=W, nsteps=30, decimation=4, warm_steps=10, options=options, qpos0=q0)
    assert rep.contact_steps > 200
    _check(rep)
