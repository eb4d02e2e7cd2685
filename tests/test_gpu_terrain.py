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
