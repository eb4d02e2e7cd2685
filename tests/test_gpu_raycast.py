"""Ray-cast sensor on the GPU against the oracle's ray casts on the same states."""
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


def _grid(nx, ny, spacing, z=0.0):
    xs = (np.arange(nx) - (nx - 1) / 2) * spacing
    ys = (np.arange(ny) - (ny - 1) / 2) * spacing
    o = np.array([[x, y, z] for x in xs for y in ys])
    return o, np.tile([0.0, 0.0, -1.0], (len(o), 1))


@pytest.mark.parametrize("name,body,world_only", [("quadruped", 1, True), ("humanoid", 1, True),
                                                  ("manipulation", 7, False)])
def test_raycast_matches_oracle(name, body, world_only):
    from oracle import Oracle, raycast as RC
    spec = getattr(I, name)()
    W = 24
    b = Batch(Model(spec), W, working_set=2)
    b.reset(6)
    ctrl = torch.tensor(I.ctrl_targets(spec, W, 20, 2), dtype=torch.float32, device="cuda")
    for t in range(20):
        b.step(ctrl[t].reshape(-1), 4)
    if name == "manipulation":
        rng = np.random.default_rng(1)
        o = rng.normal(0, 0.02, (64, 3))
        d = rng.normal(0, 1, (64, 3)) + np.array([0, 0, -2.0])
        d /= np.linalg.norm(d, axis=1, keepdims=True)
    else:
        o, d = _grid(11, 7, 0.1)
    dist = b.raycast(0, body, torch.tensor(o), torch.tensor(d), max_dist=5.0, world_only=world_only)
    dist = dist.double().cpu().numpy()
    q = b.get("qpos").view(W, spec.nq).double().cpu().numpy()
    orc = Oracle(spec)
    hits = 0
    for w in range(W):
        ref = RC.raycast(orc, spec, q[w], body, o, d, 5.0, world_only)
        np.testing.assert_allclose(dist[w], ref, atol=2e-5, rtol=1e-5)
        hits += int(np.sum(ref < 5.0))
    assert hits > W * len(o) // 4
