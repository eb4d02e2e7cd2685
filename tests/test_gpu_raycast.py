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


@pytest.mark.parametrize("name,body", [("humanoid", 30), ("manipulation", 10)])
def test_hierarchy_hits_positions_and_normals_match_oracle(name, body):
    """Rays from a body (a humanoid hand; the manipulation world's cube) toward the rest of
    the scene (every other body's geoms and the world's): the bounding-volume hierarchy
    returns exactly what testing every geom returns (distances, positions, normals), and
    both match the oracle's brute force."""
    from oracle import Oracle, raycast as RC
    spec = getattr(I, name)()
    W = 16
    b = Batch(Model(spec), W, working_set=2)
    b.reset(4)
    ctrl = torch.tensor(I.ctrl_targets(spec, W, 15, 3), dtype=torch.float32, device="cuda")
    for t in range(15):
        b.step(ctrl[t].reshape(-1), 4)
    rng = np.random.default_rng(7)
    o = rng.normal(0, 0.03, (96, 3))
    d = rng.normal(0, 1, (96, 3)) + np.array([0.0, 0.0, -0.7])     # mostly downwards, over the robot
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    hb = b.raycast_hits(0, body, torch.tensor(o), torch.tensor(d), max_dist=3.0, world_only=False)
    bf = b.raycast_hits(0, body, torch.tensor(o), torch.tensor(d), max_dist=3.0, world_only=False, hierarchy=False)
    for x, y in zip(hb, bf):
        assert torch.equal(x, y)
    dist, pos, nrm = (x.double().cpu().numpy() for x in hb)
    q = b.get("qpos").view(W, spec.nq).double().cpu().numpy()
    orc = Oracle(spec)
    hits = robot_hits = 0
    for w in range(W):
        rd, rp, rn = RC.raycast_hits(orc, spec, q[w], body, o, d, 3.0, world_only=False)
        np.testing.assert_allclose(dist[w], rd, atol=2e-5, rtol=1e-5)
        np.testing.assert_allclose(pos[w], rp, atol=5e-5)
        hit = (rd < 3.0) & (rd > 0)
        # a normal is (hit - centre) / radius: the 5e-5 m position bound over the smallest
        # radius of the scenes (0.03-0.04 m) allows about 2e-3
        np.testing.assert_allclose(nrm[w][hit], rn[hit], atol=2e-3)
        assert np.all(nrm[w][~hit] == 0.0)
        hits += int(hit.sum())
        robot_hits += int(np.sum(hit & (rp[:, 2] > 0.05)))   # above the floor: a robot or table geom
    assert hits > W * 10 and robot_hits > W


def test_height_scan_hits_on_terrain_match_oracle():
    from oracle import Oracle, raycast as RC
    spec = I.with_terrain(I.quadruped(), amplitude=0.06, seed=2)
    W = 8
    b = Batch(Model(spec), W, working_set=2)
    b.reset(8)
    ctrl = torch.tensor(I.ctrl_targets(spec, W, 10, 2), dtype=torch.float32, device="cuda")
    for t in range(10):
        b.step(ctrl[t].reshape(-1), 4)
    o, d = _grid(9, 5, 0.1, z=0.3)
    d[::3] += np.array([0.2, -0.1, 0.0])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    dist, pos, nrm = (x.double().cpu().numpy() for x in b.raycast_hits(0, 1, torch.tensor(o), torch.tensor(d),
                                                                        max_dist=3.0))
    q = b.get("qpos").view(W, spec.nq).double().cpu().numpy()
    orc = Oracle(spec)
    for w in range(W):
        rd, rp, rn = RC.raycast_hits(orc, spec, q[w], 1, o, d, 3.0, True)
        np.testing.assert_allclose(dist[w], rd, atol=3e-5, rtol=1e-5)
        np.testing.assert_allclose(pos[w], rp, atol=5e-5)
        np.testing.assert_allclose(nrm[w], rn, atol=2e-4)
        assert np.all(rn[:, 2] > 0.5)
